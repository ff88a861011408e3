"""Host-side checks that need no GPU: the C ABI library builds and exports every
entry point declared in include/qm.h, and the seeded workload generator makes
the inputs it promises."""
import ctypes
import os
import re
import subprocess

import numpy as np
import pytest
import torch

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_symbols():
    text = open(os.path.join(ROOT, "include", "qm.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(qm_[a-z0-9_]+)\s*\(", text)))


@pytest.fixture(scope="module")
def libpath():
    from paper_1507_05492_gb300 import build
    return build.build()


def test_library_exports_every_declared_symbol(libpath):
    syms = declared_symbols()
    assert len(syms) >= 15
    lib = ctypes.CDLL(libpath)
    missing = [s for s in syms if not hasattr(lib, s)]
    assert not missing, missing
    out = subprocess.run(["nm", "-D", "--defined-only", libpath], capture_output=True, text=True).stdout
    exported = set(re.findall(r" T (qm_\w+)", out))
    assert set(syms) <= exported


def test_binding_fails_loudly_without_library(monkeypatch, tmp_path):
    from paper_1507_05492_gb300 import qm
    monkeypatch.setattr(qm, "_lib", None)
    monkeypatch.setattr(qm, "LIB_PATH", str(tmp_path / "missing.so"))
    with pytest.raises(qm.LibraryMissing):
        qm.lib()


def test_strerror_without_gpu(libpath):
    lib = ctypes.CDLL(libpath)
    lib.qm_strerror.restype = ctypes.c_char_p
    assert lib.qm_strerror(0) == b"ok"
    assert lib.qm_strerror(1) == b"invalid argument"


def test_host_argument_checks_without_gpu(libpath):
    """Argument errors are reported before any device work."""
    from paper_1507_05492_gb300 import qm
    l = qm.lib()
    out = qm.QmCompare()
    a = np.zeros(1, np.int32)
    assert l.qm_compare_partitions(a.ctypes.data, a.ctypes.data, 1, 1, 1, qm.QM_HOST, ctypes.byref(out), None) \
        == qm.QM_EINVAL
    assert "n_nodes" in qm.last_error()
    h = ctypes.c_void_p()
    rp = np.array([0, 1], np.int64)
    col = np.array([0], np.int32)
    assert l.qm_load_graph(rp.ctypes.data, col.ctypes.data, 1, 1, qm.QM_HOST, 0, None, ctypes.byref(h)) \
        == qm.QM_EINVAL
    assert l.qm_load_graph(rp.ctypes.data, col.ctypes.data, 1 << 31, 2, qm.QM_HOST, 0, None, ctypes.byref(h)) \
        == qm.QM_EOVERFLOW
    # the test hooks check their arguments on the host too
    for wb, tb in ((0, 10), (17, 10), (10, 0), (10, 17)):
        assert l.qm_debug_set_perm_buckets(wb, tb, 0) == qm.QM_EINVAL, (wb, tb)
    assert l.qm_debug_set_perm_buckets(-1, -1, -1) == qm.QM_OK
    assert l.qm_debug_set_batch_wave(-1) == qm.QM_EINVAL
    assert l.qm_debug_set_batch_wave(0) == qm.QM_OK


# ------------------------------------------------------------------ generator

def test_generator_graph_is_simple_symmetric(oracle_mod):
    from paper_1507_05492_gb300 import gen
    g = gen.lfr_graph(gen.config_params("lfr10k"))
    assert g.n == 10_000 and g.row_ptr[0] == 0 and g.row_ptr[-1] == g.col.numel()
    assert oracle_mod.validate_graph(g.row_ptr.numpy(), g.col.numpy())
    deg = (g.row_ptr[1:] - g.row_ptr[:-1]).numpy()
    assert deg.max() <= 50
    assert 16.0 <= deg.mean() <= 20.5
    sizes = np.bincount(g.labels.numpy())
    assert sizes.sum() == g.n and (sizes > 0).all() and len(sizes) == g.K
    assert sizes.min() >= 20
    mu = gen.mixing_fraction(g)
    assert 0.25 <= mu <= 0.4


def test_generator_is_deterministic_and_seeded():
    from paper_1507_05492_gb300 import gen
    p = gen.LfrParams(n=3000, seed=9)
    a, b = gen.lfr_graph(p), gen.lfr_graph(p)
    assert torch.equal(a.row_ptr, b.row_ptr) and torch.equal(a.col, b.col) and torch.equal(a.labels, b.labels)
    c = gen.lfr_graph(gen.LfrParams(n=3000, seed=10))
    assert not torch.equal(a.col[:1000], c.col[:1000]) or not torch.equal(a.labels, c.labels)


def test_generator_degree_power_law_mean():
    from paper_1507_05492_gb300 import gen
    x = gen.solve_xmin(20.0, 50, 2.0)
    assert abs(x - 9.9) < 0.2          # mean of x^-2 on [x, 50] is 20
    x = gen.solve_xmin(20.0, 100, 2.0)
    assert abs(x - 7.0) < 0.1


def test_perturb_moves_exact_count():
    from paper_1507_05492_gb300 import gen
    lab = torch.randint(0, 50, (10_000,), dtype=torch.int32)
    b = gen.perturb(lab, 50, 0.1, seed=3)
    moved = (b != lab)
    assert int(moved.sum()) == 1000
    assert int(b.max()) < 50 and int(b.min()) >= 0


def test_merge_split_reaches_target():
    from paper_1507_05492_gb300 import gen
    g = gen.lfr_graph(gen.LfrParams(n=20_000, seed=4))
    for k_t in (50, g.K, 3 * g.K):
        lab, K = gen.merge_split(g.labels, k_t, seed=5)
        assert K == k_t == int(lab.max()) + 1
        assert len(np.unique(lab.numpy())) == K
    lab, K, f = gen.candidate_partition(g.labels, seed=10001)
    assert 0 <= f <= 0.5 and K == int(lab.max()) + 1


def test_bench_reads_traffic_records(tmp_path, monkeypatch):
    """bench.py takes roofline.traffic from ```json blocks of profiles/*.md (one
    record per line) and only for the current kernel sources."""
    import bench
    (tmp_path / "k.md").write_text(
        "# summary\n\n```json\n"
        '{"kernel": "k_expand", "workload": "w", "source_hash": "abc", "dram_bytes_per_launch": 123}\n'
        '{"kernel": "k_count", "workload": "w", "source_hash": "abc", "dram_bytes_per_launch": 45}\n'
        '{"kernel": "k_count", "workload": "w", "source_hash": "old", "dram_bytes_per_launch": 99}\n'
        "```\n")
    monkeypatch.setattr(bench, "PROFILE_DIR", str(tmp_path))
    monkeypatch.setattr(bench, "kernel_source_hash", lambda: "abc")
    assert bench.recorded_traffic("k_expand", "w") == 123.0
    assert bench.recorded_traffic("k_count", "w") == 45.0
    assert bench.recorded_traffic("k_count", "other") is None
    monkeypatch.setattr(bench, "kernel_source_hash", lambda: "new")
    assert bench.recorded_traffic("k_expand", "w") is None


def test_binding_checks_lengths_before_any_device_work():
    """The C ABI takes plain pointers and cannot see lengths; the binding refuses
    arrays whose shape does not match the graph (or each other) with QM_EINVAL
    before the library is called, so no kernel reads past a short buffer."""
    import types
    from paper_1507_05492_gb300 import qm
    G = types.SimpleNamespace(n=10, handle=None)     # never reaches the library
    i32 = lambda *s: np.zeros(s, np.int32)
    bad_calls = [
        (qm.score, (G, i32(9), 3)),
        (qm.score, (G, torch.zeros(1, 10, dtype=torch.int32), 3)),
        (qm.compare, (i32(5), i32(4), 1, 1)),
        (qm.score_batched, (G, i32(2, 9), 3)),
        (qm.score_batched, (G, i32(10), 3)),
        (qm.evaluate_batched, (G, i32(2, 10), 3, i32(9), 2)),
        (qm.compare_batched, (i32(10), i32(2, 9), 2, 3)),
        (qm.compare_batched, (i32(3, 9), i32(2, 9), 2, 3, False)),
        (qm.score_graphs_batched, ([G, G], [i32(10)], [3, 3])),
        (qm.score_graphs_batched, ([G, G], [i32(10), i32(11)], [3, 3])),
        (qm.score_part, (G, i32(11), 3, 0, 2)),
        (qm.autotune, (G, i32(11), 3)),
        (qm.autotune_batched, (G, i32(2, 10), 3, i32(9), 2)),
    ]
    for fn, args in bad_calls:
        with pytest.raises(qm.QmError) as e:
            fn(*args)
        assert e.value.status == qm.QM_EINVAL, fn.__name__
    with pytest.raises(qm.QmError):
        qm.Graph(np.array([0, 1, 2]), np.array([1, 0]), weights=np.ones(3, np.float32))


def test_reference_arm_sample_is_bounded():
    """--impl reference sizes its oracle sample so that warm-up plus steps stay
    within a few minutes at any step count, and never above 16M nodes."""
    import bench
    sizes = [bench.reference_sample_nodes(k, w) for k, w in ((1, 0), (2, 3), (10, 3), (50, 5), (500, 10))]
    assert sizes == sorted(sizes, reverse=True)
    assert all(1_000_000 <= n <= 16_000_000 and n % 1_000_000 == 0 for n in sizes)
    for k, w in ((10, 3), (50, 5), (100, 3)):
        n = bench.reference_sample_nodes(k, w)
        assert (k + w) * n * bench.ORACLE_S_PER_NODE <= bench.REFERENCE_BUDGET_S * 1.01


C_PROGRAM = r"""
#include "qm.h"
#include <stdio.h>
#include <string.h>
int main(void) {
    int32_t a[1] = {0};
    qm_compare out;
    qm_graph *g = NULL;
    char buf[256];
    if (strcmp(qm_strerror(QM_OK), "ok") != 0) return 1;
    /* argument errors are reported before any device work */
    if (qm_compare_partitions(a, a, 1, 1, 1, QM_HOST, &out, NULL) != QM_EINVAL) return 2;
    if (qm_last_error(buf, sizeof buf) != QM_OK || strstr(buf, "n_nodes") == NULL) return 3;
    if (qm_free_graph(g) != QM_EINVAL) return 4;            /* a null handle is refused */
    printf("%lld\n", (long long)qm_kernel_launches());
    return 0;
}
"""


def test_header_is_plain_c(libpath, tmp_path):
    """include/qm.h compiles as strict C99 (no C++ in the interface), and a C
    program links against libqm.so and gets its argument errors."""
    import shutil
    gcc = shutil.which("gcc")
    if gcc is None:
        pytest.skip("gcc not found")
    src = tmp_path / "t.c"
    src.write_text(C_PROGRAM)
    exe = tmp_path / "t"
    libdir = os.path.dirname(libpath)
    r = subprocess.run([gcc, "-std=c99", "-Wall", "-Wextra", "-pedantic", "-Werror",
                        "-I", os.path.join(ROOT, "include"), str(src), "-L", libdir, "-lqm",
                        f"-Wl,-rpath,{libdir}", "-o", str(exe)], capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
    r = subprocess.run([str(exe)], capture_output=True, text=True)
    assert r.returncode == 0, (r.returncode, r.stdout, r.stderr)
    assert r.stdout.strip() == "0"
