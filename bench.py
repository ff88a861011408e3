#!/usr/bin/env python
"""Benchmark of the community-quality library on GB300.

Headline: edges scored per second, all metrics without ground truth (Q, Qds with
its |E_ij| pair counts, the six Sec. II-B.3 measures), one qm_score_partition
call per step on a seeded LFR-style graph of 100M nodes (mean degree 20, max
100, mu = 0.3, communities of 20-1000 nodes) with its planted partition; graph
and labels resident in HBM.  Inputs (8 GB of CSR) are far larger than L2.

Also reported on the same JSON line:
  roofline      the community-major kernel's algorithmic GB/s (8|E| + 12|V| bytes
                per launch) from CUDA events around it on its own stream, against
                the measured HBM copy bandwidth;
  e2e           the same metric through the C ABI with labels in pinned host
                memory (H2D of the labels and D2H of the result in every step);
  cpu_baseline  the CPU oracle (single thread) on a bounded sample;
  extras        batched (1,024 candidates per launch, one persistent graph-
                captured kernel) vs plain per-call scoring, and the serving loop.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Under torchrun each rank scores its own replica of the workload (weak scaling,
no collective on the data path); rank 0 prints the line.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "edges scored/s (all metrics) at 100M nodes"
UNIT = "edges/s"
PEAKS_FILE = os.path.join(ROOT, "MEASURED_PEAKS.json")
PROFILE_DIR = os.path.join(ROOT, "profiles")
FALLBACK_HBM = 6800.0


# The translation units that define the kernels of the scoring step (the label
# permutation of renumbered graphs included), with the headers they include;
# the DRAM records under profiles/ name their hash.
STEP_SOURCES = ("qm_kernels.cu", "qm_community.cuh", "qm_device.cuh", "qm_finalize.cuh", "qm_expand.cuh",
                "qm_binned.cuh", "qm_weighted.cuh", "qm_internal.h", "qm_reorder.cu")


def kernel_source_hash() -> str:
    h = hashlib.sha256()
    csrc = os.path.join(ROOT, "paper_1507_05492_gb300", "csrc")
    for f in STEP_SOURCES:
        h.update(open(os.path.join(csrc, f), "rb").read())
    return h.hexdigest()[:16]


def hbm_peak():
    try:
        return float(json.load(open(PEAKS_FILE))["hbm_gbs"]), "measured"
    except Exception:
        return FALLBACK_HBM, "fallback"


def recorded_traffic(kernel: str, workload: str):
    """Per-launch DRAM bytes of `kernel` on `workload` from a committed ncu
    summary (a ```json block in profiles/*.md), or None when none matches the
    current kernel sources."""
    want = kernel_source_hash()
    try:
        names = sorted(os.listdir(PROFILE_DIR))
    except OSError:
        return None
    for f in names:
        if not f.endswith(".md"):
            continue
        text = open(os.path.join(PROFILE_DIR, f)).read()
        pos = 0
        while True:
            try:
                start = text.index("```json", pos) + len("```json")
                end = text.index("```", start)
            except ValueError:
                break
            pos = end + 3
            for line in text[start:end].splitlines():  # one JSON record per line
                try:
                    rec = json.loads(line)
                except ValueError:
                    continue
                if (rec.get("kernel") == kernel and rec.get("workload") == workload
                        and rec.get("source_hash") == want and rec.get("dram_bytes_per_launch") is not None):
                    return float(rec["dram_bytes_per_launch"])
    return None


def method_bytes(n: int, E: int) -> float:
    """The method's own bytes for one pass of all metrics without ground truth:
    per undirected edge one 4-byte endpoint id and one 4-byte label gather, per
    node an 8-byte row offset and its 4-byte label (8|E| + 12|V|).  Anything a
    pipeline writes and reads back (member lists, arc offsets, packed labels,
    keys) is overhead, not method bytes."""
    return 8.0 * E + 12.0 * n


def algorithmic_bytes(kernel: str, n: int, E: int, K: int, q: dict) -> float:
    """A kernel's share of the method bytes (method_bytes): the kernels that
    stream the adjacency with its label gathers carry all of them (they read
    every arc, every row offset and every node's label); the others carry none
    (pair counting and finalisation add no method bytes)."""
    if kernel in ("k_expand", "k_score_cm", "k_expand_half"):
        return method_bytes(n, E)
    return 0.0


def pipeline_bytes(kernel: str, n: int, E: int, K: int, q: dict) -> float:
    """Bytes a launch of `kernel` moves at minimum in this pipeline, counting
    its own intermediates (each input read once, each output written once; 4-byte
    ids and labels, 8-byte row offsets, 16-byte reciprocals).  cut = 2 x
    cut_edges_total is the number of packed inter-community entries."""
    cut = 2.0 * q["cut_edges_total"]
    table = {
        "k_score_cm": 8.0 * E + 12.0 * n,
        "k_expand": 8.0 * E + 20.0 * n + 4.0 * cut,
        "k_count": 20.0 * cut + 64.0 * K,
        "k_scatter_deg": 20.0 * n,
        "k_permute_labels": 12.0 * n,
        "k_permute_hist": 12.0 * n,
    }
    return table.get(kernel, 0.0)


def host_cpu() -> dict:
    """The host's logical CPU count and model (lscpu), recorded at run time."""
    info = {"cpu_count": os.cpu_count()}
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            k, _, v = line.partition(":")
            k, v = k.strip(), v.strip()
            if k in ("Model name", "Architecture", "Socket(s)", "Core(s) per socket", "Thread(s) per core"):
                info[k.lower().replace("(s)", "s").replace(" ", "_")] = v
    except Exception:
        pass
    try:
        info["affinity"] = len(os.sched_getaffinity(0))
    except Exception:
        pass
    return info


class Clocks:
    """nvidia-smi sampling of SM clock and throttle reasons during a timed region."""
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.path = None

    def start(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-i", str(self.gpu), "-lms", "200"], stdout=open(self.path, "w"),
                stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None
        time.sleep(0.3)

    def stop(self) -> dict:
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        try:
            for line in open(self.path):
                f = [x.strip() for x in line.split(",")]
                if len(f) < 9:
                    continue
                try:
                    sm.append(float(f[1]))
                    smax.append(float(f[2]))
                except ValueError:
                    continue
                for name, v in zip(names, f[5:9]):
                    if v.lower().startswith("active"):
                        reasons.add(name)
            os.unlink(self.path)
        except Exception:
            pass
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


# ------------------------------------------------------------------ distributed plumbing

def dist_setup(n_gpus: int):
    import torch
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    else:
        if torch.cuda.is_available():
            torch.cuda.set_device(0)
    return world, rank, local


def barrier(world):
    from paper_1507_05492_gb300 import dist as qd
    qd.barrier()


def max_over_ranks(x: float, world: int) -> float:
    from paper_1507_05492_gb300 import dist as qd
    return qd.reduce_scalar(x, "max")


def sum_over_ranks(x: float, world: int) -> float:
    from paper_1507_05492_gb300 import dist as qd
    return qd.reduce_scalar(x, "sum")


# ------------------------------------------------------------------ CPU oracle baseline

def oracle_sample(n_sample: int, device):
    """A bounded sample of the workload: the same LFR-style generator and
    parameters at n_sample nodes, planted partition."""
    from paper_1507_05492_gb300 import gen
    p = gen.config_params("lfr100m")
    p.n = n_sample
    p.seed = 303
    g = gen.lfr_graph(p, device=device)
    return g.row_ptr.cpu().numpy(), g.col.cpu().numpy(), g.labels.cpu().numpy(), g.K


def time_oracle(rp, col, lab, K, reps=1):
    from oracle import oracle
    oracle.build()
    ts = []
    for _ in range(reps):
        t0 = time.perf_counter()
        oracle.score(rp, col, lab, K)
        ts.append(time.perf_counter() - t0)
    return statistics.median(ts)


def time_oracle_all_cores(workload: str, device) -> dict:
    """The oracle's OpenMP statement (the same source built with -fopenmp) on
    the whole workload graph, all host cores, one run."""
    from oracle import oracle
    from paper_1507_05492_gb300 import gen
    try:
        oracle.build_omp()
    except Exception as e:  # reported, never silently dropped
        return {"unavailable": f"OpenMP build of the oracle failed: {e!r}"}
    g = gen.lfr_graph(gen.config_params(workload), device=device)
    rp, col, lab, K, E = g.row_ptr.cpu().numpy(), g.col.cpu().numpy(), g.labels.cpu().numpy(), g.K, g.n_edges
    del g
    t0 = time.perf_counter()
    o = oracle.score_all_cores(rp, col, lab, K)
    t = time.perf_counter() - t0
    return {"value": E / t, "unit": UNIT, "cores": o["threads"], "kind": "oracle (OpenMP build, all host cores)",
            "sample": f"the whole {workload} graph (|E| = {E}), planted partition, one run of {t:.1f} s",
            "modularity": o["modularity"]}


# ------------------------------------------------------------------ reference arm

REFERENCE_BUDGET_S = 150.0      # oracle time of a whole --impl reference run (warm-up + steps)
ORACLE_S_PER_NODE = 0.8e-6      # one oracle scoring on the workload's graph family, per node


def reference_sample_nodes(steps: int, warmup: int) -> int:
    """Sample size so that warm-up + steps oracle scorings take about
    REFERENCE_BUDGET_S: at most 16M nodes, at least 1M, whole millions."""
    n = int(REFERENCE_BUDGET_S / max(1, steps + warmup) / ORACLE_S_PER_NODE)
    return max(1_000_000, min(16_000_000, n // 1_000_000 * 1_000_000))


def run_reference(args):
    """The oracle as it stands, timed on the host cores, on a bounded sample of
    the workload (each step one oracle scoring of the sample)."""
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    import torch
    dev = "cuda" if torch.cuda.is_available() else "cpu"
    sized = args.cpu_sample_nodes is None
    if sized:
        args.cpu_sample_nodes = reference_sample_nodes(args.steps, args.warmup)
    rp, col, lab, K = oracle_sample(args.cpu_sample_nodes, dev)
    E = len(col) // 2
    for _ in range(args.warmup):
        time_oracle(rp, col, lab, K)
    ts = [time_oracle(rp, col, lab, K) for _ in range(args.steps)]
    total = sum(ts)
    value = E * args.steps / total
    sample = (f"LFR-style graph with the 100M-node workload's parameters at {args.cpu_sample_nodes} nodes "
              f"(|E| = {E}), planted partition; one oracle scoring per step"
              + (f", the sample sized so that warm-up and steps take about {REFERENCE_BUDGET_S:.0f} s" if sized
                 else ""))
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * total / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "int64+f64",
        "data": "synthetic", "config": {"workload": "lfr100m (bounded sample, see cpu_baseline)",
                                        "sample_nodes": args.cpu_sample_nodes, "n_edges": E},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle", "sample": sample,
                         "host": host_cpu()},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


# ------------------------------------------------------------------ our arm

def _timed_steps(qm, graph, labels, K, steps, stream, torch):
    """steps scoring calls on resident inputs, CUDA events on the launching
    stream; returns (ms, last result, per-step kernel traces, launches)."""
    qm.trace_enable(True)
    l0 = qm.kernel_launches()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record(stream)
    traces = []
    q = None
    for _ in range(steps):
        q = qm.score(graph, labels, K)
        traces.append(qm.trace_read())
    e1.record(stream)
    torch.cuda.synchronize()
    launches = qm.kernel_launches() - l0
    qm.trace_enable(False)
    return e0.elapsed_time(e1), q, traces, launches


def bench_headline(args, world, rank, local):
    import torch
    from paper_1507_05492_gb300 import gen, qm

    dev = torch.device("cuda", torch.cuda.current_device())
    p = gen.config_params(args.workload)
    t_gen = time.perf_counter()
    g = gen.lfr_graph(p, device=dev)
    torch.cuda.synchronize()
    t_gen = time.perf_counter() - t_gen
    t_load = time.perf_counter()
    graph = qm.Graph(g.row_ptr, g.col, reorder=not args.no_reorder)
    torch.cuda.synchronize()
    t_load = time.perf_counter() - t_load
    n, E, K = g.n, g.n_edges, g.K
    max_deg = graph.info()["max_degree"]
    labels = g.labels
    keep_csr = (g.row_ptr, g.col) if (not args.no_reorder and world == 1) else None
    del g
    torch.cuda.empty_cache()
    stream = torch.cuda.current_stream()

    if args.algorithm is not None:
        qm.set_tuning(graph, K, 512, 96 * 1024, 48, args.algorithm)
    # warm-up (also selects the launch shape)
    for _ in range(args.warmup):
        q = qm.score(graph, labels, K)
    barrier(world)
    torch.cuda.synchronize()

    clocks = Clocks(local)
    clocks.start()
    barrier(world)
    ms, q, step_kernels, launches = _timed_steps(qm, graph, labels, K, args.steps, stream, torch)
    barrier(world)
    clk = clocks.stop()
    ms_max = max_over_ranks(ms, world)
    edges_all = sum_over_ranks(float(E) * args.steps, world)
    value = edges_all / (ms_max / 1e3)

    # end to end through the C ABI with host buffers
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    lab_h = labels.cpu().pin_memory()
    for _ in range(2):
        qm.score(graph, lab_h, K)
    barrier(world)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    e0.record(stream)
    for _ in range(args.steps):
        qe = qm.score(graph, lab_h, K)
    e1.record(stream)
    torch.cuda.synchronize()
    wall = time.perf_counter() - t0
    barrier(world)
    e2e_ms = max_over_ranks(max(e0.elapsed_time(e1), wall * 1e3), world)
    assert qe == q, "host-buffer path differs from the device path"
    e2e_value = edges_all / (e2e_ms / 1e3)

    # phase B by sorting each community's run (algorithm 6) against the default
    # hashed count (algorithm 1), on the same graph and partition
    count_variants = None
    if not args.no_extras and world == 1:
        vsteps = max(1, args.steps // 2)

        def per_kernel(traces, steps):
            tot = {}
            for tr in traces:
                for name, t in tr:
                    tot[name] = tot.get(name, 0.0) + t / steps
            return {k: round(v, 3) for k, v in sorted(tot.items(), key=lambda x: -x[1])}

        qm.set_tuning(graph, K, 512, 96 * 1024, 48, 6)
        for _ in range(2):
            qm.score(graph, labels, K)
        ms6, q6, tr6, _ = _timed_steps(qm, graph, labels, K, vsteps, stream, torch)
        qm.set_tuning(graph, K, 512, 96 * 1024, 48, 1)  # the default shape again
        assert q6 == q, "sorted and hashed counts disagree"
        count_variants = {
            "what": "phase B of the two-phase pipeline: each community's packed run hashed (algorithm 1, "
                    "k_count + k_count_long) or radix-sorted and run-length counted (algorithm 6, "
                    "k_count_sort + k_count_long); same graph, partition and launch shape, identical results",
            "hash": {"ms_per_step": ms_max / args.steps, "kernel_ms": per_kernel(step_kernels, args.steps)},
            "sort": {"ms_per_step": ms6 / vsteps, "kernel_ms": per_kernel(tr6, vsteps)}}

    # metrics with ground truth at the same size: the planted partition as the
    # truth against a copy with 20% of the nodes moved (Eqs. 1-7)
    cmp = None
    if not args.no_extras and world == 1:
        found = gen.perturb(labels, K, 0.2, seed=9)
        for _ in range(2):
            qm.compare(labels, found, K, K)
        torch.cuda.synchronize()
        e0.record(stream)
        csteps = max(1, args.steps // 2)
        for _ in range(csteps):
            c = qm.compare(labels, found, K, K)
        e1.record(stream)
        torch.cuda.synchronize()
        cms = e0.elapsed_time(e1) / csteps
        cmp = {"what": "planted partition (truth) vs 20% of nodes moved (found), all seven indices",
               "ms_per_call": cms, "nodes_per_s": n / (cms / 1e3), "nmi": c["nmi"], "ari": c["ari"]}
        del found

    # the paper's detected-vs-truth workload at this size: detect C' with the
    # device label propagation, then score C' and compare it with the truth
    detect = None
    if not args.no_extras and world == 1:
        rounds = 10
        qm.label_propagation(graph, 1)
        torch.cuda.synchronize()
        e0.record(stream)
        found, k_found = qm.label_propagation(graph, rounds)
        e1.record(stream)
        torch.cuda.synchronize()
        t_lpa = e0.elapsed_time(e1)
        e0.record(stream)
        qd = qm.score(graph, found, k_found)
        cd = qm.compare(labels, found, K, k_found)
        e1.record(stream)
        torch.cuda.synchronize()
        detect = {"what": f"label propagation ({rounds} rounds) on the graph, then all metrics of C' "
                          "with and without the planted truth",
                  "lpa_ms": t_lpa, "lpa_ms_per_round": t_lpa / rounds, "score_and_compare_ms": e0.elapsed_time(e1),
                  "k_found": k_found, "nmi": cd["nmi"], "ari": cd["ari"], "f_measure": cd["f_measure"],
                  "modularity": qd["modularity"]}
        del found

    # the same workload on the graph as given (no reorder), for comparison
    unordered = None
    if keep_csr is not None:
        g2 = qm.Graph(*keep_csr)
        for _ in range(2):
            qm.score(g2, labels, K)
        ms2, q2, tr2, _ = _timed_steps(qm, g2, labels, K, max(1, args.steps // 2), stream, torch)
        assert q2 == q, "reordered and unordered graphs disagree"
        st2 = max(1, args.steps // 2)
        unordered = {"value": E * st2 / (ms2 / 1e3), "unit": UNIT, "ms_per_step": ms2 / st2,
                     "kernel_ms": {k: round(sum(t for nm, t in tr if nm == k) / st2, 3)
                                   for k in sorted({nm for tr in tr2 for nm, _ in tr})
                                   for tr in [sum(tr2, [])]}}
        g2.close()
        del keep_csr, g2
        torch.cuda.empty_cache()

    peak, peak_kind = hbm_peak()
    kernel_shares = {}
    for tr in step_kernels:
        for name, t in tr:
            kernel_shares[name] = kernel_shares.get(name, 0.0) + t
    total_k = sum(kernel_shares.values()) or 1.0
    # the dominant kernel: largest share of the step's kernel time (one launch per step)
    top = max(kernel_shares, key=kernel_shares.get)
    top_avg = kernel_shares[top] / args.steps
    b_alg = algorithmic_bytes(top, n, E, K, q)
    achieved = b_alg / (top_avg / 1e3) / 1e9
    b_step = method_bytes(n, E)
    top_traffic = recorded_traffic(top, args.workload)
    # whole-pass DRAM traffic from the committed ncu records of every kernel of
    # the step (null when any record is missing or the kernels changed since)
    launches_per_step = {}
    for tr in step_kernels:
        for name, _ in tr:
            launches_per_step[name] = launches_per_step.get(name, 0) + 1
    pass_bytes = 0.0
    for name, cnt in launches_per_step.items():
        rec = recorded_traffic(name, args.workload)
        if rec is None:
            pass_bytes = None
            break
        pass_bytes += rec * cnt / args.steps
    res = dict(
        value=value, ms_per_step=ms_max / args.steps, launches=launches,
        e2e={"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": 4 * n,
             "d2h_bytes_per_step": 4 + 120},
        roofline={"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                  "frac": achieved / peak, "traffic": top_traffic,
                  "kernel": top, "peak_kind": f"{peak_kind} (burst copy)",
                  "algorithmic_bytes_per_launch": b_alg, "kernel_ms": top_avg,
                  "bytes_rule": "method bytes 8|E| + 12|V| per pass, carried by the kernel that streams "
                                "the adjacency with its label gathers",
                  "overfetch": (top_traffic / b_alg) if (top_traffic and b_alg) else None,
                  "pipeline_bytes_per_launch": pipeline_bytes(top, n, E, K, q),
                  "traffic_source": "dram__bytes_read.sum + dram__bytes_write.sum per launch from the committed "
                                    "ncu record of this kernel and workload (profiles/), null unless its "
                                    "source hash matches the current kernel sources",
                  "step_algorithmic_bytes": b_step,
                  "step_algorithmic_gbs": b_step / (ms_max / args.steps / 1e3) / 1e9,
                  "step_dram_bytes": pass_bytes,
                  "step_dram_gbs": (pass_bytes / (ms_max / args.steps / 1e3) / 1e9) if pass_bytes else None,
                  "step_dram_frac": (pass_bytes / (ms_max / args.steps / 1e3) / 1e9 / peak) if pass_bytes else None,
                  "step_algorithmic_frac": b_step / (ms_max / args.steps / 1e3) / 1e9 / peak},
        clocks=clk,
        config={"workload": f"{args.workload}: LFR-style, n={n}, |E|={E}, K={K}, max degree {max_deg}, "
                            f"mean degree 20 target, mu=0.3, communities 20-1000, planted partition",
                "n_nodes": n, "n_edges": E, "n_communities": K, "seed": p.seed,
                "graph_load": ("QM_REORDER: label-propagation renumbering at load, "
                               f"{t_load:.2f} s incl. copy (not in the timed region)") if not args.no_reorder
                              else f"as given, {t_load:.2f} s",
                "l2": "inputs (CSR 8 GB + labels 0.4 GB) far larger than the 129 MB L2",
                "generation_s": round(t_gen, 1)},
        kernel_share={k: round(v / total_k, 4) for k, v in sorted(kernel_shares.items(), key=lambda x: -x[1])},
        result={k: q[k] for k in ("modularity", "modularity_density", "mean_conductance",
                                  "n_community_pairs", "cut_edges_total")},
        unordered=unordered,
        compare=cmp,
        detect=detect,
        count_variants=count_variants,
    )
    graph.close()
    del labels, lab_h
    torch.cuda.empty_cache()
    return res


def bench_batched(args):
    """1,024 candidate partitions of 100k-node graphs (mu 0.1 / 0.3 / 0.5): one
    persistent graph-captured launch per graph (all metrics with and without
    ground truth) against the plain loop of one score + one compare call each."""
    import torch
    from paper_1507_05492_gb300 import gen, qm
    dev = torch.device("cuda", torch.cuda.current_device())
    out = {}
    for name in ("lfr100k_mu01", "lfr100k_mu03", "lfr100k_mu05"):
        g = gen.lfr_graph(gen.config_params(name), device=dev)
        graph = qm.Graph(g.row_ptr, g.col)
        t0 = time.perf_counter()
        labs, Ks = gen.candidate_batch(g.labels, args.batch, seed=10_000)
        t_cand = time.perf_counter() - t0
        truth = g.labels
        # launch shape picked by the batched autotuner on a quarter of the batch (set-up, untimed)
        qsub = max(1, args.batch // 4)
        tuned = qm.autotune_batched(graph, labs[:qsub], Ks[:qsub], truth, g.K)
        qm.set_batch_tuning(graph, max(Ks), tuned["threads"], tuned["smem_bytes"], tuned["big_community"])
        for _ in range(2):
            oq, oc = qm.evaluate_batched(graph, labs, Ks, truth, g.K)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        reps = 3
        for _ in range(reps):
            oq, oc = qm.evaluate_batched(graph, labs, Ks, truth, g.K)
        t_b = (time.perf_counter() - t0) / reps
        # the plain loop over the same candidates (and a bit-for-bit check)
        n_plain = min(args.batch, args.plain_sample)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        same = True
        for p in range(n_plain):
            pq = qm.score(graph, labs[p], Ks[p])
            pc = qm.compare(truth, labs[p], g.K, Ks[p])
            same &= (pq == oq[p]) and (pc == oc[p])
        t_p = (time.perf_counter() - t0) / n_plain
        out[name] = {"partitions_per_s_batched": args.batch / t_b,
                     "partitions_per_s_plain": 1.0 / t_p,
                     "speedup": (args.batch / t_b) * t_p,
                     "ms_per_launch": t_b * 1e3, "identical_to_plain": bool(same),
                     "plain_checked": n_plain, "K_range": [int(min(Ks)), int(max(Ks))],
                     "candidate_generation_s": round(t_cand, 1),
                     "tuned_shape": {k: tuned[k] for k in ("threads", "smem_bytes", "big_community")},
                     "edge_scorings_per_s": args.batch * g.n_edges / t_b}
        graph.close()
        del g, labs
        torch.cuda.empty_cache()
    return out


def bench_configs(args):
    """The smaller configurations, one plain call each: 10k nodes (scoring of
    the planted partition and its comparison with a 10% perturbed copy; latency
    bound, so microseconds per call) and 10M nodes (scoring of the planted
    partition; ms per call and edges/s).  CUDA events on the current stream,
    median of the timed calls."""
    import torch
    from paper_1507_05492_gb300 import gen, qm
    dev = torch.device("cuda", torch.cuda.current_device())
    stream = torch.cuda.current_stream()
    out = {}

    def timed(fn, reps):
        for _ in range(3):
            fn()
        ts = []
        for _ in range(reps):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            torch.cuda.synchronize()
            e0.record(stream)
            fn()
            e1.record(stream)
            torch.cuda.synchronize()
            ts.append(e0.elapsed_time(e1))
        return statistics.median(ts)

    g = gen.lfr_graph(gen.config_params("lfr10k"), device=dev)
    graph = qm.Graph(g.row_ptr, g.col)
    b = gen.perturb(g.labels, g.K, 0.1, seed=101)
    t_s = timed(lambda: qm.score(graph, g.labels, g.K), 20)
    t_c = timed(lambda: qm.compare(g.labels, b, g.K, g.K), 20)
    out["lfr10k"] = {"score_us_per_call": 1e3 * t_s, "compare_us_per_call": 1e3 * t_c,
                     "n_edges": g.n_edges}
    graph.close()
    g = gen.lfr_graph(gen.config_params("lfr10m"), device=dev)
    for reorder in (True, False):
        graph = qm.Graph(g.row_ptr, g.col, reorder=reorder)
        t = timed(lambda: qm.score(graph, g.labels, g.K), 10)
        out["lfr10m" + ("" if reorder else "_graph_as_given")] = {
            "score_ms_per_call": t, "edges_per_s": g.n_edges / (t / 1e3)}
        graph.close()
    # batched candidates at this size: 16 perturbed copies of the planted partition (0-50% of
    # the nodes moved), each scored and compared with the planted one, in one batched call
    # (above 2^21 nodes the plain pipelines of every item, captured into one launch) against
    # the plain loop of one score and one compare call each
    P = 16
    cands = torch.stack([gen.perturb(g.labels, g.K, 0.5 * p / (P - 1), seed=900 + p) for p in range(P)])
    Ks = [g.K] * P
    graph = qm.Graph(g.row_ptr, g.col, reorder=True)

    def plain_loop():
        return [(qm.score(graph, cands[p], g.K), qm.compare(g.labels, cands[p], g.K, g.K)) for p in range(P)]
    t_b = timed(lambda: qm.evaluate_batched(graph, cands, Ks, g.labels, g.K), 5)
    t_p = timed(plain_loop, 5)
    oq, oc = qm.evaluate_batched(graph, cands, Ks, g.labels, g.K)
    same = all(oq[p] == a and oc[p] == b for p, (a, b) in enumerate(plain_loop()))
    out["lfr10m_batched_candidates"] = {"candidates": P, "ms_per_batch": t_b, "partitions_per_s_batched": P / (t_b / 1e3),
                                        "partitions_per_s_plain": P / (t_p / 1e3), "identical_to_plain": bool(same),
                                        "what": "score + compare with the planted partition per candidate, graph reordered"}
    graph.close()
    del cands
    # the same graph with a float32 weight per edge (a hash of the pair, in [0.05, 5))
    u = torch.repeat_interleave(torch.arange(g.n, device=dev), g.row_ptr[1:] - g.row_ptr[:-1])
    v = g.col.to(torch.int64)
    a, b = torch.minimum(u, v), torch.maximum(u, v)
    h = (a * 2654435761 + b * 40503 + 12345) % (1 << 32)
    w = (0.05 + h.to(torch.float64) / float(1 << 32) * 4.95).to(torch.float32)
    del u, v, a, b, h
    graph = qm.Graph(g.row_ptr, g.col, reorder=True, weights=w)
    t = timed(lambda: qm.score(graph, g.labels, g.K), 5)
    out["lfr10m_weighted"] = {"score_ms_per_call": t, "edges_per_s": g.n_edges / (t / 1e3),
                              "what": "weighted Q and Qds (edge weights, unweighted densities), graph reordered"}
    graph.close()
    del w
    del g
    torch.cuda.empty_cache()
    return out


def bench_serving(args):
    from paper_1507_05492_gb300 import server
    return server.run_benchmark(duration_s=args.serve_seconds, rate=args.serve_rate, seed=11)


def run_compare_only(args):
    """Metrics with ground truth alone on the workload (Eqs. 1-7): the planted
    partition against a copy with 20% of the nodes moved, and against itself;
    one JSON line with ms per call (CUDA events on the current stream)."""
    import torch
    import __graft_entry__
    __graft_entry__.build()
    from paper_1507_05492_gb300 import gen, qm
    dev = torch.device("cuda", torch.cuda.current_device())
    g = gen.lfr_graph(gen.config_params(args.workload), device=dev)
    stream = torch.cuda.current_stream()
    out = {"workload": args.workload, "n_nodes": g.n, "k": g.K}
    found = gen.perturb(g.labels, g.K, 0.2, seed=9)
    for name, f in (("vs_20pct_moved", found), ("vs_itself", g.labels)):
        for _ in range(args.warmup):
            qm.compare(g.labels, f, g.K, g.K)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(args.steps):
            c = qm.compare(g.labels, f, g.K, g.K)
        e1.record(stream)
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / args.steps
        out[name] = {"ms_per_call": ms, "nodes_per_s": g.n / (ms / 1e3), "n_cells": c["n_cells"],
                     "nmi": c["nmi"], "ari": c["ari"]}
    print(json.dumps(out), flush=True)
    return 0


def run_batched_only(args):
    """The batched launch alone (all metrics with and without ground truth of
    --batch candidates of the 100k-node, mu = 0.3 graph) with the default
    launch shape; one JSON line with partitions/s (CUDA events)."""
    import torch
    import __graft_entry__
    __graft_entry__.build()
    from paper_1507_05492_gb300 import gen, qm
    dev = torch.device("cuda", torch.cuda.current_device())
    g = gen.lfr_graph(gen.config_params("lfr100k_mu03"), device=dev)
    graph = qm.Graph(g.row_ptr, g.col)
    labs, Ks = gen.candidate_batch(g.labels, args.batch, seed=10_000)
    stream = torch.cuda.current_stream()
    for _ in range(args.warmup):
        qm.evaluate_batched(graph, labs, Ks, g.labels, g.K)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(args.steps):
        qm.evaluate_batched(graph, labs, Ks, g.labels, g.K)
    e1.record(stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / args.steps
    print(json.dumps({"workload": "lfr100k_mu03", "candidates": args.batch, "ms_per_launch": ms,
                      "partitions_per_s": args.batch / (ms / 1e3), "tuning": qm.get_batch_tuning(graph, max(Ks))}),
          flush=True)
    return 0


def run_ours(args):
    import torch
    world, rank, local = dist_setup(args.gpus)
    import __graft_entry__
    __graft_entry__.build()
    res = bench_headline(args, world, rank, local)
    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        if args.cpu_sample_nodes is None:
            args.cpu_sample_nodes = 16_000_000   # one oracle scoring, about 12 s
        rp, col, lab, K = oracle_sample(args.cpu_sample_nodes, torch.device("cuda", local))
        t = time_oracle(rp, col, lab, K, reps=1)
        E = len(col) // 2
        cpu = {"value": E / t, "unit": UNIT, "cores": 1, "kind": "oracle",
               "sample": f"LFR-style graph with the workload's parameters at {args.cpu_sample_nodes} nodes "
                         f"(|E| = {E}), planted partition, single-threaded oracle, {t:.1f} s",
               "host": host_cpu()}
        del rp, col, lab
        cpu["all_cores"] = time_oracle_all_cores(args.workload, torch.device("cuda", local))
    extras = {}
    if rank == 0 and world == 1 and not args.no_extras:
        try:
            extras["batched"] = bench_batched(args)
        except Exception as e:  # reported, never silently dropped
            extras["batched"] = {"error": repr(e)}
        try:
            extras["configs"] = bench_configs(args)
        except Exception as e:
            extras["configs"] = {"error": repr(e)}
        try:
            extras["serving"] = bench_serving(args)
        except Exception as e:
            extras["serving"] = {"error": repr(e)}
    if rank == 0:
        line = {
            "metric": METRIC, "value": res["value"], "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": res["ms_per_step"],
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "int64 counts + f64 (128-bit fixed-point sums)", "data": "synthetic",
            "config": res["config"] | {"parallelism": f"replicas x{world}"},
            "roofline": res["roofline"], "cpu_baseline": cpu, "e2e": res["e2e"],
            "gpu_launches": res["launches"], "clocks": res["clocks"],
            "kernel_share": res["kernel_share"], "result": res["result"],
            "orders": {"reordered" if not args.no_reorder else "as_given":
                       {"value": res["value"], "unit": UNIT, "ms_per_step": res["ms_per_step"]}}
                      | ({"as_given": res["unordered"]} if res["unordered"] else {}),
            "extras": extras | ({"compare": res["compare"]} if res["compare"] else {})
                      | ({"detect": res["detect"]} if res["detect"] else {})
                      | ({"count_variants": res["count_variants"]} if res["count_variants"] else {}),
        }
        print(json.dumps(line), flush=True)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--workload", default="lfr100m")
    ap.add_argument("--cpu-sample-nodes", type=int, default=None,
                    help="nodes of the oracle's sample (default: 16M for cpu_baseline; for --impl reference, "
                         "sized so that warm-up + steps take about 150 s)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-extras", action="store_true")
    ap.add_argument("--no-reorder", action="store_true",
                    help="load the graph as given instead of with QM_REORDER")
    ap.add_argument("--batch", type=int, default=1024)
    ap.add_argument("--plain-sample", type=int, default=256)
    ap.add_argument("--serve-seconds", type=float, default=60.0)
    ap.add_argument("--serve-rate", type=float, default=200.0)
    ap.add_argument("--only-compare", action="store_true",
                    help="time only the metrics with ground truth (Eqs. 1-7) on the workload")
    ap.add_argument("--only-batched", action="store_true",
                    help="time only the batched launch (--batch candidates, default launch shape)")
    ap.add_argument("--algorithm", type=int, default=None,
                    help="score with this tuning algorithm (include/qm.h; default launch shape) instead of "
                         "the untuned default")
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    if args.impl == "reference":
        return run_reference(args)
    if args.only_compare:
        return run_compare_only(args)
    if args.only_batched:
        return run_batched_only(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
