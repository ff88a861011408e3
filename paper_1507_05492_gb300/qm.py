"""Python binding of libqm.so (include/qm.h): argument marshalling only.

Every metric is computed by the CUDA kernels behind the C ABI; this module only
converts tensors/arrays to pointers and C structs to dicts.  There is no CPU
fallback: if the library is not built, every call raises ``LibraryMissing``.

Low-level functions carry the C names (``qm_load_graph``, ``qm_score_partition``
...).  The ``Graph`` class and the ``score`` / ``compare`` / ``evaluate_batched``
helpers wrap them for tensors.
"""
from __future__ import annotations

import ctypes
import os
import threading

import numpy as np
import torch

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_build", "libqm.so")

QM_OK, QM_EINVAL, QM_ENOMEM, QM_ECUDA, QM_ETIMEOUT, QM_EOVERFLOW, QM_EBUSY = range(7)
QM_HOST, QM_DEVICE = 0, 1
QM_VALIDATE = 1
QM_REORDER = 2
QM_SHARED_TRUTH = 1


class LibraryMissing(RuntimeError):
    pass


class QmError(RuntimeError):
    def __init__(self, status: int, where: str, detail: str):
        super().__init__(f"{where}: status {status} ({detail})")
        self.status = status


class QmQuality(ctypes.Structure):
    _fields_ = [(n, ctypes.c_int64) for n in (
        "n_nodes", "n_edges", "n_communities_nonempty", "intra_edges_total", "cut_edges_total",
        "n_community_pairs", "pair_count_sq_sum")] + [(n, ctypes.c_double) for n in (
        "modularity", "modularity_density", "mean_intra_edges", "mean_intra_density",
        "mean_contraction", "mean_inter_edges", "mean_expansion", "mean_conductance")]


class QmCompare(ctypes.Structure):
    _fields_ = [(n, ctypes.c_int64) for n in (
        "n_nodes", "k_truth", "k_found", "n_cells", "a11", "a10", "a01", "a00", "nvd_sum")] + [
        (n, ctypes.c_double) for n in ("vi", "nmi", "f_measure", "nvd", "ri", "ari", "ji")]


PARTIAL_WORDS = 32


class QmPartial(ctypes.Structure):
    _fields_ = [("n_nodes", ctypes.c_int64), ("n_edges", ctypes.c_int64), ("nranks", ctypes.c_int32),
                ("flags", ctypes.c_int32), ("ranks_mask", ctypes.c_uint64),
                ("words", ctypes.c_uint64 * PARTIAL_WORDS)]


class QmPercomm(ctypes.Structure):
    _fields_ = [(n, ctypes.c_void_p) for n in (
        "size", "intra_edges", "inter_edges", "intra_density", "contraction", "expansion",
        "conductance", "qds_term")]


class QmTraceEvent(ctypes.Structure):
    _fields_ = [("name", ctypes.c_char * 28), ("ms", ctypes.c_float)]


class QmTuning(ctypes.Structure):
    _fields_ = [(n, ctypes.c_int32) for n in ("threads", "smem_bytes", "big_community", "blocks_per_sm",
                                                    "algorithm")]


_lib = None
_lock = threading.Lock()
_P = ctypes.c_void_p
_I64 = ctypes.c_int64
_I32 = ctypes.c_int32


def _signatures(lib):
    S = ctypes.c_int
    table = {
        "qm_load_graph": [_P, _P, _I64, _I64, S, ctypes.c_uint, _P, ctypes.POINTER(_P)],
        "qm_free_graph": [_P],
        "qm_graph_info": [_P, _P, _P, _P, _P],
        "qm_score_partition": [_P, _P, _I32, S, _P, _P, _P],
        "qm_compare_partitions": [_P, _P, _I64, _I32, _I32, S, _P, _P],
        "qm_score_partitions_batched": [_P, _P, _I32, _P, S, _P, _P],
        "qm_compare_partitions_batched": [_P, _P, _I64, _I32, _P, _P, ctypes.c_uint, S, _P, _P],
        "qm_evaluate_partitions_batched": [_P, _P, _I32, _P, _P, _I32, S, _P, _P, _P],
        "qm_score_graphs_batched": [_P, _P, _P, _I32, S, _P, _P],
        "qm_workspace_bytes": [_P, _I32, _I32, _I32, _P],
        "qm_release_cache": [],
        "qm_debug_set_stage_wait": [_I64],
        "qm_debug_set_batch_wave": [_I32],
        "qm_debug_set_perm_buckets": [_I32, _I32, _I64],
        "qm_score_cover": [_P, _P, _P, _I32, S, _P, _P],
        "qm_compare_covers": [_P, _P, _I32, _P, _P, _I32, _I64, S, _P, _P],
        "qm_autotune": [_P, _P, _I32, S, _P, _P],
        "qm_get_tuning": [_P, _I32, _P],
        "qm_set_tuning": [_P, _I32, _P],
        "qm_autotune_batched": [_P, _P, _I32, _P, _P, _I32, S, _P, _P],
        "qm_label_propagation": [_P, _I32, _P, S, _P, _P],
        "qm_load_graph_weighted": [_P, _P, _P, _I64, _I64, S, ctypes.c_uint, _P, ctypes.POINTER(_P)],
        "qm_score_partition_part": [_P, _P, _I32, S, _I32, _I32, _P, _P],
        "qm_partials_combine": [_P, _I32, _P],
        "qm_partial_finalize": [_P, _P, _P],
        "qm_get_batch_tuning": [_P, _I32, _P],
        "qm_set_batch_tuning": [_P, _I32, _P],
        "qm_last_error": [_P, ctypes.c_size_t],
        "qm_trace_enable": [_I32],
        "qm_trace_read": [_P, _I32, _P],
    }
    for name, args in table.items():
        f = getattr(lib, name)
        f.argtypes = args
        f.restype = ctypes.c_int
    lib.qm_strerror.argtypes = [ctypes.c_int]
    lib.qm_strerror.restype = ctypes.c_char_p
    lib.qm_kernel_launches.argtypes = []
    lib.qm_kernel_launches.restype = ctypes.c_int64


def lib():
    """The loaded libqm.so; raises LibraryMissing when it has not been built."""
    global _lib
    if _lib is not None:
        return _lib
    with _lock:
        if _lib is None:
            if not os.path.exists(LIB_PATH):
                raise LibraryMissing(f"{LIB_PATH} is not built; run __graft_entry__.build() "
                                     "or python -m paper_1507_05492_gb300.build")
            l = ctypes.CDLL(LIB_PATH)
            _signatures(l)
            _lib = l
    return _lib


def last_error() -> str:
    buf = ctypes.create_string_buffer(512)
    lib().qm_last_error(buf, 512)
    return buf.value.decode(errors="replace")


def _check(rc: int, where: str):
    if rc != QM_OK:
        raise QmError(rc, where, last_error())


def kernel_launches() -> int:
    return int(lib().qm_kernel_launches())


# ------------------------------------------------------------------ marshalling

def _stream_ptr(stream) -> int | None:
    if stream is None:
        if torch.cuda.is_available() and torch.cuda.is_initialized():
            return torch.cuda.current_stream().cuda_stream or None
        return None
    if isinstance(stream, torch.cuda.Stream):
        return stream.cuda_stream or None
    return int(stream) or None


def _labels_arg(x, name="labels"):
    """Returns (pointer, memory kind, keep-alive object) for an int32 label array."""
    if isinstance(x, torch.Tensor):
        if x.dtype != torch.int32 or not x.is_contiguous():
            raise TypeError(f"{name} must be a contiguous int32 tensor")
        return x.data_ptr(), (QM_DEVICE if x.is_cuda else QM_HOST), x
    a = np.ascontiguousarray(np.asarray(x), dtype=np.int32)
    return a.ctypes.data, QM_HOST, a


def _cover_arg(cover, n, where_name):
    """(mptr pointer, memb pointer, memory kind, keep-alive, m) of a cover given
    as (mptr int64[n + 1], memb int32[m]), both torch tensors on one device or
    both host arrays.  The lengths are checked here (the C ABI cannot see them)."""
    mptr, memb = cover
    if isinstance(mptr, torch.Tensor) or isinstance(memb, torch.Tensor):
        _need(isinstance(mptr, torch.Tensor) and isinstance(memb, torch.Tensor) and mptr.device == memb.device,
              where_name, "mptr and memb must both be tensors on one device, or both host arrays")
        _need(mptr.dtype == torch.int64 and memb.dtype == torch.int32 and mptr.is_contiguous() and
              memb.is_contiguous(), where_name, "mptr must be contiguous int64 and memb contiguous int32")
        _need(tuple(mptr.shape) == (n + 1,), where_name, f"mptr of shape {tuple(mptr.shape)} for {n} nodes")
        m = int(mptr[-1].item())
        _need(memb.dim() == 1 and memb.numel() >= m, where_name, f"memb holds {memb.numel()} ids, mptr[n] = {m}")
        return mptr.data_ptr(), memb.data_ptr(), (QM_DEVICE if mptr.is_cuda else QM_HOST), (mptr, memb), m
    mp = np.ascontiguousarray(np.asarray(mptr), dtype=np.int64)
    mb = np.ascontiguousarray(np.asarray(memb), dtype=np.int32)
    _need(mp.shape == (n + 1,), where_name, f"mptr of shape {mp.shape} for {n} nodes")
    m = int(mp[-1]) if n >= 0 else 0
    _need(mb.ndim == 1 and mb.size >= m, where_name, f"memb holds {mb.size} ids, mptr[n] = {m}")
    if mb.size == 0:
        mb = np.zeros(1, np.int32)
    return mp.ctypes.data, mb.ctypes.data, QM_HOST, (mp, mb), m


def _shape(x) -> tuple:
    return tuple(x.shape)


def _need(ok: bool, where: str, detail: str):
    """Lengths the C ABI cannot see (it takes plain pointers) are checked here,
    before any device work: a short buffer would otherwise be read past its end."""
    if not ok:
        raise QmError(QM_EINVAL, where, detail)


def _struct_dict(s) -> dict:
    return {name: getattr(s, name) for name, _ in s._fields_}


# ------------------------------------------------------------------ graph

class Graph:
    """A symmetric CSR graph resident on the current CUDA device."""

    def __init__(self, row_ptr, col, validate: bool = False, reorder: bool = False, stream=None, weights=None):
        """reorder=True stores the graph renumbered for locality (QM_REORDER):
        calls still take labels in the caller's node order and give the same
        results.  weights (float32 per arc, in the memory of col) loads a
        weighted graph (qm_load_graph_weighted)."""
        if isinstance(row_ptr, torch.Tensor):
            rp = row_ptr.contiguous().to(torch.int64)
            cl = col.contiguous().to(torch.int32)
            where = QM_DEVICE if rp.is_cuda else QM_HOST
            if (where == QM_DEVICE) != cl.is_cuda:
                raise ValueError("row_ptr and col must live in the same memory")
            keep = (rp, cl)
            prp, pcl = rp.data_ptr(), cl.data_ptr()
            n, arcs = rp.numel() - 1, cl.numel()
            if weights is not None:
                wt = torch.as_tensor(weights).to(device=cl.device, dtype=torch.float32).contiguous()
                _need(wt.numel() == arcs, "qm_load_graph_weighted", f"{wt.numel()} weights for {arcs} arcs")
                keep = keep + (wt,)
                pwt = wt.data_ptr()
        else:
            rp = np.ascontiguousarray(row_ptr, dtype=np.int64)
            cl = np.ascontiguousarray(col, dtype=np.int32)
            keep = (rp, cl)
            prp, pcl = rp.ctypes.data, cl.ctypes.data
            where = QM_HOST
            n, arcs = len(rp) - 1, len(cl)
            if weights is not None:
                wt = np.ascontiguousarray(np.asarray(weights), dtype=np.float32)
                _need(wt.size == arcs, "qm_load_graph_weighted", f"{wt.size} weights for {arcs} arcs")
                keep = keep + (wt,)
                pwt = wt.ctypes.data
        h = ctypes.c_void_p()
        flags = (QM_VALIDATE if validate else 0) | (QM_REORDER if reorder else 0)
        if weights is None:
            _check(lib().qm_load_graph(prp, pcl, n, arcs, where, flags, _stream_ptr(stream), ctypes.byref(h)),
                   "qm_load_graph")
        else:
            _check(lib().qm_load_graph_weighted(prp, pcl, pwt, n, arcs, where, flags, _stream_ptr(stream),
                                                ctypes.byref(h)), "qm_load_graph_weighted")
        del keep
        self.handle = h
        self.n = n
        self.n_arcs = arcs
        self.n_edges = arcs // 2
        self.reordered = reorder
        self.weighted = weights is not None

    @classmethod
    def from_csr(cls, row_ptr, col, **kwargs) -> "Graph":
        """The same as Graph(row_ptr, col, ...): a symmetric CSR from torch tensors
        (host or device) or numpy arrays."""
        return cls(row_ptr, col, **kwargs)

    def info(self) -> dict:
        vals = [ctypes.c_int64() for _ in range(3)]
        nbytes = ctypes.c_size_t()
        _check(lib().qm_graph_info(self.handle, *[ctypes.byref(v) for v in vals], ctypes.byref(nbytes)),
               "qm_graph_info")
        return dict(n_nodes=vals[0].value, n_edges=vals[1].value, max_degree=vals[2].value,
                    device_bytes=nbytes.value)

    def close(self):
        if getattr(self, "handle", None):
            lib().qm_free_graph(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


# ------------------------------------------------------------------ calls

def score(graph: Graph, labels, K: int, per_community: bool = False, stream=None) -> dict:
    """qm_score_partition: Q, Qds and the six measures of one partition."""
    ptr, where, keep = _labels_arg(labels)
    _need(_shape(keep) == (graph.n,), "qm_score_partition", f"labels of shape {_shape(keep)} for {graph.n} nodes")
    out = QmQuality()
    pc = None
    arrays = None
    if per_community:
        dev = where == QM_DEVICE
        mk = (lambda dt: torch.empty(K, dtype=dt, device=labels.device)) if dev else \
            (lambda dt: np.empty(K, dtype=np.int64 if dt is torch.int64 else np.float64))
        names = ["size", "intra_edges", "inter_edges", "intra_density", "contraction", "expansion",
                 "conductance", "qds_term"]
        arrays = {k: mk(torch.int64 if i < 3 else torch.float64) for i, k in enumerate(names)}
        ptrs = [(a.data_ptr() if dev else a.ctypes.data) for a in arrays.values()]
        pc = QmPercomm(*ptrs)
    rc = lib().qm_score_partition(graph.handle, ptr, int(K), where, ctypes.byref(out),
                                  ctypes.byref(pc) if pc is not None else None, _stream_ptr(stream))
    del keep
    _check(rc, "qm_score_partition")
    d = _struct_dict(out)
    if arrays is not None:
        d["per_community"] = arrays
    return d


def score_cover(graph: "Graph", cover, K: int, stream=None) -> dict:
    """qm_score_cover: Q, Qds and the six measures of a cover (overlapping
    communities): cover = (mptr int64[n + 1], memb int32[m]), the communities of
    node u being memb[mptr[u]:mptr[u + 1]] in increasing order.  The field
    cut_edges_total holds the sum over communities of |E_c^out|."""
    mp, mb, where, keep, _ = _cover_arg(cover, graph.n, "qm_score_cover")
    out = QmQuality()
    rc = lib().qm_score_cover(graph.handle, mp, mb, int(K), where, ctypes.byref(out), _stream_ptr(stream))
    del keep
    _check(rc, "qm_score_cover")
    return _struct_dict(out)


def compare_covers(truth, k_truth: int, found, k_found: int, n: int, stream=None) -> dict:
    """qm_compare_covers: Eqs. (1)-(7) for two covers of n nodes, each given as
    (mptr, memb) like score_cover; truth first."""
    ap, am, wa, ka_keep, _ = _cover_arg(truth, n, "qm_compare_covers")
    bp, bm, wb, kb_keep, _ = _cover_arg(found, n, "qm_compare_covers")
    _need(wa == wb, "qm_compare_covers", "both covers must be in the same kind of memory")
    out = QmCompare()
    rc = lib().qm_compare_covers(ap, am, int(k_truth), bp, bm, int(k_found), int(n), wa, ctypes.byref(out),
                                 _stream_ptr(stream))
    del ka_keep, kb_keep
    _check(rc, "qm_compare_covers")
    return _struct_dict(out)


def compare(truth, found, k_truth: int, k_found: int, stream=None) -> dict:
    """qm_compare_partitions: Eqs. (1)-(7) for ground truth ``truth`` and detected ``found``."""
    pt, wt, kt_ = _labels_arg(truth, "truth")
    pf, wf, kf_ = _labels_arg(found, "found")
    if wt != wf:
        raise ValueError("truth and found must live in the same memory")
    n = kt_.numel() if isinstance(kt_, torch.Tensor) else len(kt_)
    _need(_shape(kt_) == (n,) and _shape(kf_) == (n,), "qm_compare_partitions",
          f"truth of shape {_shape(kt_)} and found of shape {_shape(kf_)}")
    out = QmCompare()
    rc = lib().qm_compare_partitions(pt, pf, n, int(k_truth), int(k_found), wt, ctypes.byref(out),
                                     _stream_ptr(stream))
    _check(rc, "qm_compare_partitions")
    return _struct_dict(out)


def _k_array(K, P):
    k = np.ascontiguousarray(np.broadcast_to(np.asarray(K, dtype=np.int32), (P,)))
    return k


def score_batched(graph: Graph, labels, K, stream=None) -> list[dict]:
    """qm_score_partitions_batched over a [P, n] int32 label matrix."""
    ptr, where, keep = _labels_arg(labels)
    _need(len(_shape(keep)) == 2 and _shape(keep)[1] == graph.n, "qm_score_partitions_batched",
          f"labels of shape {_shape(keep)} for {graph.n} nodes")
    P = _shape(keep)[0]
    k = _k_array(K, P)
    out = (QmQuality * P)()
    _check(lib().qm_score_partitions_batched(graph.handle, ptr, P, k.ctypes.data, where, out,
                                             _stream_ptr(stream)), "qm_score_partitions_batched")
    return [_struct_dict(o) for o in out]


def evaluate_batched(graph: Graph, labels, K, truth, k_truth: int, stream=None):
    """qm_evaluate_partitions_batched: (quality list, compare list) for P candidates."""
    ptr, where, keep = _labels_arg(labels)
    pt, wt, keep_t = _labels_arg(truth, "truth")
    if wt != where:
        raise ValueError("labels and truth must live in the same memory")
    _need(len(_shape(keep)) == 2 and _shape(keep)[1] == graph.n and _shape(keep_t) == (graph.n,),
          "qm_evaluate_partitions_batched",
          f"labels of shape {_shape(keep)} and truth of shape {_shape(keep_t)} for {graph.n} nodes")
    P = _shape(keep)[0]
    k = _k_array(K, P)
    oq = (QmQuality * P)()
    oc = (QmCompare * P)()
    _check(lib().qm_evaluate_partitions_batched(graph.handle, ptr, P, k.ctypes.data, pt, int(k_truth), where,
                                                oq, oc, _stream_ptr(stream)), "qm_evaluate_partitions_batched")
    return [_struct_dict(o) for o in oq], [_struct_dict(o) for o in oc]


def compare_batched(truth, found, k_truth, k_found, shared_truth: bool = True, stream=None) -> list[dict]:
    """qm_compare_partitions_batched over a [P, n] detected-label matrix."""
    pf, wf, keep_f = _labels_arg(found, "found")
    pt, wt, keep_t = _labels_arg(truth, "truth")
    if wt != wf:
        raise ValueError("truth and found must live in the same memory")
    _need(len(_shape(keep_f)) == 2, "qm_compare_partitions_batched", f"found of shape {_shape(keep_f)}")
    P, n = _shape(keep_f)
    _need(_shape(keep_t) == ((n,) if shared_truth else (P, n)), "qm_compare_partitions_batched",
          f"truth of shape {_shape(keep_t)} for found of shape {(P, n)}")
    kt = _k_array(k_truth, 1 if shared_truth else P)
    kf = _k_array(k_found, P)
    out = (QmCompare * P)()
    _check(lib().qm_compare_partitions_batched(pt, pf, n, P, kt.ctypes.data, kf.ctypes.data,
                                               QM_SHARED_TRUTH if shared_truth else 0, wf, out,
                                               _stream_ptr(stream)), "qm_compare_partitions_batched")
    return [_struct_dict(o) for o in out]


def score_graphs_batched(graphs: list[Graph], labels: list, K: list[int], stream=None) -> list[dict]:
    """qm_score_graphs_batched: one partition on each of several graphs."""
    count = len(graphs)
    _need(len(labels) == count and len(K) == count, "qm_score_graphs_batched",
          f"{count} graphs, {len(labels)} label arrays, {len(K)} label counts")
    args = [_labels_arg(l) for l in labels]
    for i, (g, a) in enumerate(zip(graphs, args)):
        _need(_shape(a[2]) == (g.n,), "qm_score_graphs_batched",
              f"labels {i} of shape {_shape(a[2])} for {g.n} nodes")
    kinds = {a[1] for a in args}
    if len(kinds) != 1:
        raise ValueError("all label arrays must live in the same memory")
    gs = (ctypes.c_void_p * count)(*[g.handle.value for g in graphs])
    ls = (ctypes.c_void_p * count)(*[a[0] for a in args])
    k = np.ascontiguousarray(K, dtype=np.int32)
    out = (QmQuality * count)()
    _check(lib().qm_score_graphs_batched(gs, ls, k.ctypes.data, count, kinds.pop(), out, _stream_ptr(stream)),
           "qm_score_graphs_batched")
    return [_struct_dict(o) for o in out]


def workspace_bytes(graph: Graph, K: int, k_truth: int | None = None) -> int:
    b = ctypes.c_size_t()
    _check(lib().qm_workspace_bytes(graph.handle, int(K), 1 if k_truth else 0, int(k_truth or 0),
                                    ctypes.byref(b)), "qm_workspace_bytes")
    return b.value


def autotune(graph: Graph, labels, K: int, stream=None) -> dict:
    ptr, where, keep = _labels_arg(labels)
    _need(_shape(keep) == (graph.n,), "qm_autotune", f"labels of shape {_shape(keep)} for {graph.n} nodes")
    t = QmTuning()
    _check(lib().qm_autotune(graph.handle, ptr, int(K), where, _stream_ptr(stream), ctypes.byref(t)),
           "qm_autotune")
    return _struct_dict(t)


def get_tuning(graph: Graph, K: int) -> dict:
    t = QmTuning()
    _check(lib().qm_get_tuning(graph.handle, int(K), ctypes.byref(t)), "qm_get_tuning")
    return _struct_dict(t)


def set_tuning(graph: Graph, K: int, threads: int, smem_bytes: int, big_community: int, algorithm: int = 1):
    """algorithm 0: one-kernel community pass; 1: expand + count (two phases); 2-5: variants of 1's
    gathers; 6: as 1 with a sort + run-length count of each community's labels; 7: as 1 with each
    undirected edge gathered once (include/qm.h)."""
    t = QmTuning(threads, smem_bytes, big_community, 0, algorithm)
    _check(lib().qm_set_tuning(graph.handle, int(K), ctypes.byref(t)), "qm_set_tuning")


def score_part(graph: Graph, labels, K: int, rank: int, nranks: int, stream=None) -> QmPartial:
    """qm_score_partition_part: the exact partial sums of shard `rank` of
    `nranks` (communities c with c mod nranks == rank, Sec. III-A)."""
    ptr, where, keep = _labels_arg(labels)
    _need(_shape(keep) == (graph.n,), "qm_score_partition_part", f"labels of shape {_shape(keep)} for {graph.n} nodes")
    out = QmPartial()
    rc = lib().qm_score_partition_part(graph.handle, ptr, int(K), where, int(rank), int(nranks),
                                       ctypes.byref(out), _stream_ptr(stream))
    del keep
    _check(rc, "qm_score_partition_part")
    return out


def combine_parts(parts) -> QmPartial:
    """qm_partials_combine: exact sum of partials (host only, no GPU needed)."""
    parts = list(parts)
    arr = (QmPartial * len(parts))(*parts)
    out = QmPartial()
    _check(lib().qm_partials_combine(arr, len(parts), ctypes.byref(out)), "qm_partials_combine")
    return out


def finalize_part(part: QmPartial, stream=None) -> dict:
    """qm_partial_finalize: the metrics of a partial that covers every shard."""
    out = QmQuality()
    _check(lib().qm_partial_finalize(ctypes.byref(part), ctypes.byref(out), _stream_ptr(stream)),
           "qm_partial_finalize")
    return _struct_dict(out)


def part_to_array(part: QmPartial) -> np.ndarray:
    """The partial as int64[4 + PARTIAL_WORDS] (for transport between processes)."""
    head = np.array([part.n_nodes, part.n_edges, part.nranks | (part.flags << 32), 0], np.int64)
    head[3] = np.array([part.ranks_mask], np.uint64).view(np.int64)[0]
    words = np.frombuffer(bytes(part.words), dtype=np.uint64).view(np.int64)
    return np.concatenate([head, words])


def part_from_array(a) -> QmPartial:
    a = np.ascontiguousarray(np.asarray(a, dtype=np.int64))
    p = QmPartial()
    p.n_nodes, p.n_edges = int(a[0]), int(a[1])
    p.nranks, p.flags = int(a[2]) & 0xFFFFFFFF, int(a[2]) >> 32
    p.ranks_mask = int(a[3:4].view(np.uint64)[0])
    ctypes.memmove(p.words, a[4:4 + PARTIAL_WORDS].view(np.uint64).tobytes(), 8 * PARTIAL_WORDS)
    return p


def label_propagation(graph: Graph, rounds: int = 10, device: bool = True, stream=None):
    """qm_label_propagation: (labels int32[n] (cuda tensor, or numpy when
    device=False), K')."""
    if device:
        out = torch.empty(graph.n, dtype=torch.int32, device="cuda")
        ptr, where = out.data_ptr(), QM_DEVICE
    else:
        out = np.empty(graph.n, dtype=np.int32)
        ptr, where = out.ctypes.data, QM_HOST
    k = ctypes.c_int32()
    _check(lib().qm_label_propagation(graph.handle, int(rounds), ptr, where, ctypes.byref(k),
                                      _stream_ptr(stream)), "qm_label_propagation")
    return out, int(k.value)


def autotune_batched(graph: Graph, labels, K, truth=None, k_truth: int = 0, stream=None) -> dict:
    """qm_autotune_batched over a [P, n] label matrix (and an optional truth)."""
    ptr, where, keep = _labels_arg(labels)
    _need(len(_shape(keep)) == 2 and _shape(keep)[1] == graph.n, "qm_autotune_batched",
          f"labels of shape {_shape(keep)} for {graph.n} nodes")
    pt = None
    if truth is not None:
        pt, wt, keep_t = _labels_arg(truth, "truth")
        if wt != where:
            raise ValueError("labels and truth must live in the same memory")
        _need(_shape(keep_t) == (graph.n,), "qm_autotune_batched", f"truth of shape {_shape(keep_t)}")
    P = _shape(keep)[0]
    k = _k_array(K, P)
    t = QmTuning()
    _check(lib().qm_autotune_batched(graph.handle, ptr, P, k.ctypes.data, pt, int(k_truth), where,
                                     _stream_ptr(stream), ctypes.byref(t)), "qm_autotune_batched")
    return _struct_dict(t)


def get_batch_tuning(graph: Graph, K: int) -> dict:
    t = QmTuning()
    _check(lib().qm_get_batch_tuning(graph.handle, int(K), ctypes.byref(t)), "qm_get_batch_tuning")
    return _struct_dict(t)


def set_batch_tuning(graph: Graph, K: int, threads: int, smem_bytes: int, big_community: int):
    t = QmTuning(threads, smem_bytes, big_community, 0, 0)
    _check(lib().qm_set_batch_tuning(graph.handle, int(K), ctypes.byref(t)), "qm_set_batch_tuning")


def trace_enable(on: bool = True):
    """Per-thread kernel timing with CUDA events on the launching stream."""
    _check(lib().qm_trace_enable(1 if on else 0), "qm_trace_enable")


def trace_read() -> list[tuple[str, float]]:
    """(kernel name, device ms) of every kernel of the calling thread's last traced call."""
    cap = 64
    buf = (QmTraceEvent * cap)()
    n = ctypes.c_int32()
    _check(lib().qm_trace_read(buf, cap, ctypes.byref(n)), "qm_trace_read")
    return [(buf[i].name.decode(), float(buf[i].ms)) for i in range(min(n.value, cap))]


def release_cache():
    _check(lib().qm_release_cache(), "qm_release_cache")


def debug_set_batch_wave(items: int):
    """qm_debug_set_batch_wave: cap the batched pipeline's waves at `items`
    items for later calls (0: automatic).  A test hook for the wave loop."""
    _check(lib().qm_debug_set_batch_wave(int(items)), "qm_debug_set_batch_wave")


def debug_set_perm_buckets(window_bits: int = -1, tile_bits: int = -1, min_nodes: int = -1):
    """qm_debug_set_perm_buckets: graphs loaded with QM_REORDER afterwards
    bring labels into their node order in two passes (tiles of 2**tile_bits
    caller ids, windows of 2**window_bits new ids) when they have more than
    min_nodes nodes (negative: the defaults, automatic bits and 2**24).  A test hook
    for the two-pass permutation."""
    _check(lib().qm_debug_set_perm_buckets(int(window_bits), int(tile_bits), int(min_nodes)),
           "qm_debug_set_perm_buckets")


def debug_set_stage_wait(polls: int):
    """qm_debug_set_stage_wait: poll limit of the pair-count kernel's staging
    wait for later calls (0: every such wait expires at once; negative: the
    default).  A test hook for the QM_ETIMEOUT path."""
    _check(lib().qm_debug_set_stage_wait(int(polls)), "qm_debug_set_stage_wait")
