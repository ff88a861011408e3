"""ctypes wrapper of the plain CPU oracle in ``qm_oracle.c``.

TEST INFRASTRUCTURE ONLY: imported by ``tests/``, by the smoke check and by the
benchmark's CPU-baseline leg.  The product library never imports this module and
this module never imports the product library.

Each function returns plain Python/numpy values.  The metric definitions and the
readings of the paper taken where it is silent are stated in ``qm_oracle.c``.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "qm_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "liboracle.so")
_OMP_PATH = os.path.join(_BUILD, "liboracle_omp.so")
_lock = threading.Lock()
_lib = None
_omp = None

SCORE_DBL = ["modularity", "modularity_density", "mean_intra_edges", "mean_intra_density",
             "mean_contraction", "mean_inter_edges", "mean_expansion", "mean_conductance",
             "cond_modularity", "cond_modularity_density"]
SCORE_I64 = ["n_nodes", "n_edges", "n_communities_nonempty", "intra_edges_total",
             "cut_edges_total", "n_community_pairs", "pair_count_sq_sum"]
COMPARE_DBL = ["vi", "nmi", "f_measure", "nvd", "ri", "ari", "ji",
               "cond_vi", "cond_nmi_num", "nmi_den_abs"]
COMPARE_I64 = ["n_nodes", "k_truth", "k_found", "n_cells", "a11", "a10", "a01", "a00", "nvd_sum"]


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (no FMA contraction) and return the .so path."""
    with _lock:
        if (not force and os.path.exists(_LIB_PATH)
                and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC)):
            return _LIB_PATH
        os.makedirs(_BUILD, exist_ok=True)
        tmp = _LIB_PATH + f".tmp{os.getpid()}"
        subprocess.run(["gcc", "-std=c11", "-O2", "-fPIC", "-shared", "-ffp-contract=off",
                        "-o", tmp, _SRC, "-lm"], check=True)
        os.replace(tmp, _LIB_PATH)
        return _LIB_PATH


def build_omp(force: bool = False) -> str:
    """The same source built with OpenMP (-fopenmp) for the all-core timed
    baseline (oq_score_omp); returns the .so path."""
    with _lock:
        if (not force and os.path.exists(_OMP_PATH)
                and os.path.getmtime(_OMP_PATH) >= os.path.getmtime(_SRC)):
            return _OMP_PATH
        os.makedirs(_BUILD, exist_ok=True)
        tmp = _OMP_PATH + f".tmp{os.getpid()}"
        subprocess.run(["gcc", "-std=c11", "-O2", "-fPIC", "-shared", "-ffp-contract=off", "-fopenmp",
                        "-o", tmp, _SRC, "-lm"], check=True)
        os.replace(tmp, _OMP_PATH)
        return _OMP_PATH


def _load_omp():
    global _omp
    if _omp is None:
        lib = ctypes.CDLL(build_omp())
        p = ctypes.c_void_p
        lib.oq_score_omp.argtypes = [p, p, ctypes.c_int64, p, ctypes.c_int32, p, p, p]
        lib.oq_score_omp.restype = ctypes.c_int
        _omp = lib
    return _omp


def score_all_cores(row_ptr, col, labels, K: int) -> dict:
    """Eqs. (8)-(9) and the six measures with OpenMP threads over the host cores
    (the same quantities as score() without per-community arrays); the result
    carries the thread count in "threads"."""
    row_ptr = _as(row_ptr, np.int64)
    col = _as(col, np.int32)
    labels = _as(labels, np.int32)
    n = len(row_ptr) - 1
    assert len(labels) == n
    dbl = np.zeros(16, np.float64)
    i64 = np.zeros(8, np.int64)
    th = np.zeros(1, np.int32)
    _check(_load_omp().oq_score_omp(_ptr(row_ptr), _ptr(col), n, _ptr(labels), int(K), _ptr(dbl), _ptr(i64),
                                    _ptr(th)), "score_all_cores")
    out = {k: float(dbl[i]) for i, k in enumerate(SCORE_DBL)}
    out.update({k: int(i64[i]) for i, k in enumerate(SCORE_I64)})
    out["threads"] = int(th[0])
    return out


def _load():
    global _lib
    if _lib is not None:
        return _lib
    lib = ctypes.CDLL(build())
    p = ctypes.c_void_p
    i64 = ctypes.c_int64
    i32 = ctypes.c_int32
    lib.oq_validate_graph.argtypes = [p, p, i64]
    lib.oq_score.argtypes = [p, p, i64, p, i32, p, p] + [p] * 8
    lib.oq_compare.argtypes = [p, p, i64, i32, i32, p, p]
    lib.oq_pairs_bruteforce.argtypes = [p, p, i64, p]
    lib.oq_compare_bruteforce.argtypes = [p, p, i64, i32, i32, p]
    lib.oq_score_bruteforce.argtypes = [p, p, i64, p, i32, p]
    lib.oq_score_communities.argtypes = [p, p, i64, p, i32, p, i64, p, p]
    lib.oq_label_propagation.argtypes = [p, p, i64, i32, p, p]
    lib.oq_score_weighted.argtypes = [p, p, p, i64, p, i32, p]
    lib.oq_validate_cover.argtypes = [p, p, i64, i32]
    lib.oq_score_cover.argtypes = [p, p, i64, p, p, i32, p, p]
    lib.oq_compare_cover.argtypes = [p, p, i32, p, p, i32, i64, p, p]
    lib.oq_pairs_cover_bruteforce.argtypes = [p, p, p, p, i64, p]
    for f in (lib.oq_validate_graph, lib.oq_score, lib.oq_compare, lib.oq_pairs_bruteforce,
              lib.oq_compare_bruteforce, lib.oq_score_bruteforce, lib.oq_score_communities,
              lib.oq_label_propagation, lib.oq_score_weighted, lib.oq_validate_cover, lib.oq_score_cover,
              lib.oq_compare_cover, lib.oq_pairs_cover_bruteforce):
        f.restype = ctypes.c_int
    _lib = lib
    return lib


class OracleError(RuntimeError):
    pass


def _ptr(a: np.ndarray):
    return ctypes.c_void_p(a.ctypes.data)


def _as(a, dtype):
    return np.ascontiguousarray(np.asarray(a), dtype=dtype)


def _check(rc: int, what: str):
    if rc != 0:
        raise OracleError(f"oracle {what} failed with code {rc}")


def validate_graph(row_ptr, col) -> bool:
    row_ptr = _as(row_ptr, np.int64)
    col = _as(col, np.int32)
    return _load().oq_validate_graph(_ptr(row_ptr), _ptr(col), len(row_ptr) - 1) == 0


def score(row_ptr, col, labels, K: int, per_community: bool = False) -> dict:
    """Eqs. (8)-(9) and the six measures of Sec. II-B.3 for one partition."""
    row_ptr = _as(row_ptr, np.int64)
    col = _as(col, np.int32)
    labels = _as(labels, np.int32)
    n = len(row_ptr) - 1
    assert len(labels) == n
    dbl = np.zeros(16, np.float64)
    i64 = np.zeros(8, np.int64)
    pcs = None
    if per_community:
        pcs = {k: np.zeros(K, np.int64) for k in ("size", "intra_edges", "inter_edges")}
        pcs.update({k: np.zeros(K, np.float64) for k in ("intra_density", "contraction",
                                                         "expansion", "conductance", "qds_term")})
        arrs = [_ptr(pcs[k]) for k in ("size", "intra_edges", "inter_edges", "intra_density",
                                       "contraction", "expansion", "conductance", "qds_term")]
    else:
        arrs = [None] * 8
    rc = _load().oq_score(_ptr(row_ptr), _ptr(col), n, _ptr(labels), int(K), _ptr(dbl), _ptr(i64),
                          *arrs)
    _check(rc, "score")
    out = {k: float(dbl[i]) for i, k in enumerate(SCORE_DBL)}
    out.update({k: int(i64[i]) for i, k in enumerate(SCORE_I64)})
    if pcs is not None:
        out["per_community"] = pcs
    return out


def compare(truth, found, k_truth: int, k_found: int) -> dict:
    """Eqs. (1)-(7) for ground truth C = ``truth`` and detected C' = ``found``."""
    a = _as(truth, np.int32)
    b = _as(found, np.int32)
    assert len(a) == len(b)
    dbl = np.zeros(16, np.float64)
    i64 = np.zeros(16, np.int64)
    rc = _load().oq_compare(_ptr(a), _ptr(b), len(a), int(k_truth), int(k_found), _ptr(dbl), _ptr(i64))
    _check(rc, "compare")
    out = {k: float(dbl[i]) for i, k in enumerate(COMPARE_DBL)}
    out.update({k: int(i64[i]) for i, k in enumerate(COMPARE_I64)})
    return out


def pairs_bruteforce(truth, found) -> tuple[int, int, int, int]:
    """Algorithm 4: (a11, a10, a01, a00) by visiting every node pair."""
    a = _as(truth, np.int32)
    b = _as(found, np.int32)
    out = np.zeros(4, np.int64)
    _check(_load().oq_pairs_bruteforce(_ptr(a), _ptr(b), len(a), _ptr(out)), "pairs_bruteforce")
    return tuple(int(x) for x in out)


def compare_bruteforce(truth, found, k_truth: int, k_found: int) -> dict:
    """Set-intersection evaluation of Eqs. (1)-(4)."""
    a = _as(truth, np.int32)
    b = _as(found, np.int32)
    dbl = np.zeros(4, np.float64)
    _check(_load().oq_compare_bruteforce(_ptr(a), _ptr(b), len(a), int(k_truth), int(k_found),
                                         _ptr(dbl)), "compare_bruteforce")
    return dict(vi=float(dbl[0]), nmi=float(dbl[1]), f_measure=float(dbl[2]), nvd=float(dbl[3]))


def score_bruteforce(row_ptr, col, labels, K: int) -> dict:
    """Community-pair scan evaluation of Eqs. (8)-(9)."""
    row_ptr = _as(row_ptr, np.int64)
    col = _as(col, np.int32)
    labels = _as(labels, np.int32)
    dbl = np.zeros(2, np.float64)
    _check(_load().oq_score_bruteforce(_ptr(row_ptr), _ptr(col), len(row_ptr) - 1, _ptr(labels),
                                       int(K), _ptr(dbl)), "score_bruteforce")
    return dict(modularity=float(dbl[0]), modularity_density=float(dbl[1]))


def score_communities(row_ptr, col, labels, K: int, ids) -> dict:
    """Per-community values of Eq. (9) and Sec. II-B.3 for the sampled ids only."""
    row_ptr = _as(row_ptr, np.int64)
    col = _as(col, np.int32)
    labels = _as(labels, np.int32)
    ids = _as(ids, np.int32)
    m = len(ids)
    i64 = np.zeros((m, 4), np.int64)
    dbl = np.zeros((m, 2), np.float64)
    _check(_load().oq_score_communities(_ptr(row_ptr), _ptr(col), len(row_ptr) - 1, _ptr(labels), int(K),
                                        _ptr(ids), m, _ptr(i64), _ptr(dbl)), "score_communities")
    return dict(size=i64[:, 0], intra_edges=i64[:, 1], inter_edges=i64[:, 2], distinct_neighbours=i64[:, 3],
                qds_term=dbl[:, 0], split=dbl[:, 1])


def score_weighted(row_ptr, col, weight, labels, K: int) -> dict:
    """Eqs. (8)-(9) on a weighted graph: edge amounts weighted, densities
    unweighted (the paper's note on the weighted case)."""
    row_ptr = _as(row_ptr, np.int64)
    col = _as(col, np.int32)
    weight = _as(weight, np.float64)
    labels = _as(labels, np.int32)
    dbl = np.zeros(5, np.float64)
    _check(_load().oq_score_weighted(_ptr(row_ptr), _ptr(col), _ptr(weight), len(row_ptr) - 1, _ptr(labels),
                                     int(K), _ptr(dbl)), "score_weighted")
    return dict(modularity=float(dbl[0]), modularity_density=float(dbl[1]), cond_modularity=float(dbl[2]),
                cond_modularity_density=float(dbl[3]), total_weight=float(dbl[4]))


def label_propagation(row_ptr, col, rounds: int):
    """Synchronous label propagation (the detector family of Sec. I and IV-C):
    (labels renumbered to [0, K'), K')."""
    row_ptr = _as(row_ptr, np.int64)
    col = _as(col, np.int32)
    n = len(row_ptr) - 1
    out = np.zeros(n, np.int32)
    k = np.zeros(1, np.int32)
    _check(_load().oq_label_propagation(_ptr(row_ptr), _ptr(col), n, int(rounds), _ptr(out), _ptr(k)),
           "label_propagation")
    return out, int(k[0])


def within(gpu: float, ref: float, cond: float = 0.0, rel: float = 1e-12) -> bool:
    """Tolerance rule: |g - o| <= rel * max(|o|, conditioning)."""
    return abs(gpu - ref) <= rel * max(abs(ref), abs(cond), 1e-300)


# ------------------------------------------------------------------ covers (overlapping communities)

def cover_from_lists(lists):
    """(mptr int64[n+1], memb int32[...]) from one list of community ids per node
    (each list sorted, without repeats)."""
    mptr = np.zeros(len(lists) + 1, np.int64)
    mptr[1:] = np.cumsum([len(x) for x in lists])
    memb = np.array([c for x in lists for c in x], dtype=np.int32)
    return mptr, memb


def validate_cover(mptr, memb, K: int) -> bool:
    mptr = _as(mptr, np.int64)
    memb = _as(memb, np.int32) if len(memb) else np.zeros(1, np.int32)
    return _load().oq_validate_cover(_ptr(mptr), _ptr(memb), len(mptr) - 1, int(K)) == 0


def score_cover(row_ptr, col, mptr, memb, K: int) -> dict:
    """Eqs. (8)-(9) and the six measures for a cover (the set formulas read
    literally, see qm_oracle.c); cut_edges_total holds the sum over communities
    of |E_c^out|."""
    row_ptr = _as(row_ptr, np.int64)
    col = _as(col, np.int32)
    mptr = _as(mptr, np.int64)
    memb = _as(memb, np.int32) if len(memb) else np.zeros(1, np.int32)
    dbl = np.zeros(16, np.float64)
    i64 = np.zeros(8, np.int64)
    _check(_load().oq_score_cover(_ptr(row_ptr), _ptr(col), len(row_ptr) - 1, _ptr(mptr), _ptr(memb), int(K),
                                  _ptr(dbl), _ptr(i64)), "score_cover")
    out = {k: float(dbl[i]) for i, k in enumerate(SCORE_DBL)}
    out.update({k: int(i64[i]) for i, k in enumerate(SCORE_I64)})
    return out


def compare_cover(aptr, amemb, ka: int, bptr, bmemb, kb: int) -> dict:
    """Eqs. (1)-(7) for two covers (ground truth first)."""
    aptr, bptr = _as(aptr, np.int64), _as(bptr, np.int64)
    amemb = _as(amemb, np.int32) if len(amemb) else np.zeros(1, np.int32)
    bmemb = _as(bmemb, np.int32) if len(bmemb) else np.zeros(1, np.int32)
    assert len(aptr) == len(bptr)
    dbl = np.zeros(16, np.float64)
    i64 = np.zeros(16, np.int64)
    _check(_load().oq_compare_cover(_ptr(aptr), _ptr(amemb), int(ka), _ptr(bptr), _ptr(bmemb), int(kb),
                                    len(aptr) - 1, _ptr(dbl), _ptr(i64)), "compare_cover")
    out = {k: float(dbl[i]) for i, k in enumerate(COMPARE_DBL)}
    out.update({k: int(i64[i]) for i, k in enumerate(COMPARE_I64)})
    return out


def pairs_cover_bruteforce(aptr, amemb, bptr, bmemb) -> tuple[int, int, int, int]:
    """(a11, a10, a01, a00) of two covers by visiting every node pair."""
    aptr, bptr = _as(aptr, np.int64), _as(bptr, np.int64)
    amemb = _as(amemb, np.int32) if len(amemb) else np.zeros(1, np.int32)
    bmemb = _as(bmemb, np.int32) if len(bmemb) else np.zeros(1, np.int32)
    out = np.zeros(4, np.int64)
    _check(_load().oq_pairs_cover_bruteforce(_ptr(aptr), _ptr(amemb), _ptr(bptr), _ptr(bmemb), len(aptr) - 1,
                                             _ptr(out)), "pairs_cover_bruteforce")
    return tuple(int(x) for x in out)
