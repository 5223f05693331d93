"""CPU-only checks of the C-ABI library: it builds for sm_103a, loads, exports
every entry point include/nr.h declares, and its host-side pieces (the
quadrature rule, argument validation without a device) behave.  No kernel is
launched here."""
import ctypes
import math
import os
import re

import numpy as np
import pytest

import oracle
import paper_2509_06924_gb300 as nr
from paper_2509_06924_gb300 import workloads as W

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def header_functions():
    text = open(os.path.join(ROOT, "include", "nr.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"^\s*(?:nr_status|void|const char \*)\s*\*?\s*(nr_\w+)\s*\(", text, re.M)))


def test_library_builds_and_exports_every_declared_symbol():
    lib = nr.load_library()
    declared = header_functions()
    assert len(declared) >= 10, declared
    for name in declared:
        assert hasattr(lib, name), f"{name} declared in nr.h but not exported"
    assert set(declared) == set(nr.EXPORTS)


@pytest.mark.parametrize("K", list(range(1, 33)))
def test_library_quadrature_matches_numpy(K):
    x, w = nr.quadrature(K)
    xr, wr = np.polynomial.hermite.hermgauss(K)
    np.testing.assert_allclose(x, xr, rtol=0, atol=1e-12 * max(1, np.abs(xr).max()))
    np.testing.assert_allclose(w, wr, rtol=1e-10, atol=1e-15)
    assert abs(w.sum() - math.sqrt(math.pi)) < 1e-13


def test_library_and_oracle_quadratures_agree():
    # two independent constructions (Jacobi eigenvalues + Newton vs bisection
    # + Newton; derivative vs Christoffel weights)
    for K in (17, 21, 32):
        x1, w1 = nr.quadrature(K)
        x2, w2 = oracle.gauss_hermite(K)
        np.testing.assert_allclose(x1, x2, rtol=0, atol=5e-13)
        np.testing.assert_allclose(w1, w2, rtol=1e-11, atol=1e-16)


def test_quadrature_rejects_bad_order():
    lib = nr.load_library()
    x = np.zeros(64)
    w = np.zeros(64)
    for K in (0, -3, nr.MAX_QUAD + 1):
        st = lib.nr_quadrature(K, x.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
                               w.ctypes.data_as(ctypes.POINTER(ctypes.c_double)))
        assert st == nr.NR_EINVAL
        assert b"outside" in lib.nr_last_error()


def test_null_arguments_are_rejected_without_a_device():
    lib = nr.load_library()
    assert lib.nr_create(None, None) == nr.NR_EINVAL
    assert lib.nr_loglik(None, None, None, None) == nr.NR_EINVAL
    assert lib.nr_plan(None, None) == nr.NR_EINVAL
    lib.nr_destroy(None)  # no-op


def test_release_library_refuses_the_debug_hook():
    """nr_debug_poison_plan exists only in NR_DEBUG builds: the release
    library answers NR_EINVAL before touching anything."""
    lib = nr.load_library()
    assert not nr.debug_build_selected()
    assert lib.nr_debug_poison_plan(None, None, 1) == nr.NR_EINVAL
    assert b"NR_DEBUG" in lib.nr_last_error()


def test_create_without_gpu_fails_cleanly():
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    lib = nr.load_library()
    h = ctypes.c_void_p()
    st = lib.nr_create(ctypes.byref(h), None)
    assert st in (nr.NR_ECUDA, nr.NR_ENOMEM)
    assert h.value is None
    assert len(lib.nr_last_error()) > 0


def test_context_refuses_without_gpu():
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    with pytest.raises(RuntimeError):
        nr.Context()


def test_struct_layouts_match_header():
    # nr_options: 8 int32; nr_batch: 2 int32, 3 pointers, 2 int32, 5 pointers
    assert ctypes.sizeof(nr.Options) == 32
    assert ctypes.sizeof(nr.CBatch) == 8 + 3 * 8 + 8 + 5 * 8


# ------------------------------------------------------------- workloads ----
def test_workloads_are_seeded_and_shaped():
    a = W.make_workload("thick_oxide", n_stacks=10)
    b = W.make_workload("thick_oxide", n_stacks=10)
    np.testing.assert_array_equal(a.params, b.params)
    assert a.n_stacks == 10 and a.n_quad == 21 and int(a.q_off[-1]) == 400
    assert a.evals == 10 * 400 * 21
    L = W.layout(1)
    d = a.params.reshape(10, 10)[:, L["d"]]
    assert np.all((d >= 1000) & (d <= 3000))
    c = W.make_workload("thick_oxide", n_stacks=10, seed_offset=1)
    assert not np.array_equal(a.params, c.params)
    full = W.make_workload("thick_oxide")
    assert full.evals == 16384 * 400 * 21


def test_contrast_workload_structure():
    wl = W.make_workload("oled_cofit", n_stacks=2)
    assert wl.n_stacks == 6 and list(wl.dataset) == [0, 1, 2, 0, 1, 2]
    assert list(np.diff(wl.q_off)) == [150, 220, 300]
    P = W.n_params(10)
    p = wl.params.reshape(6, P)
    L = W.layout(10)
    # layer parameters shared across the three contrasts of a chain
    np.testing.assert_array_equal(p[0, L["d"]], p[2, L["d"]])
    assert p[1, L["rho"]][0] == 6.35e-6 and p[2, L["rho"]][-1] == 4.2e-6


def test_uneven_workload_ranges():
    wl = W.make_workload("uneven", n_stacks=200)
    assert wl.n_layers.min() >= 1 and wl.n_layers.max() <= 20
    lens = np.diff(wl.q_off)
    assert lens.min() >= 50 and lens.max() <= 500
    rel = wl.dq / wl.q
    assert rel.min() >= 0.0199 and rel.max() <= 0.0801


def test_golden_data_match_grids():
    for name in ("film_1l", "thick_oxide", "oled_cofit", "vi_step"):
        wl = W.make_workload(name, n_stacks=1)
        assert np.all(wl.r_err > 0) and np.all(wl.r_obs > 0)


# ----------------------------------------------------------------- bench ----
def test_flop_table_is_monotone_and_positive():
    import bench
    f = [bench.flops_per_eval(n, 21) for n in range(0, 21)]
    assert all(x > 0 for x in f)
    assert all(b > a for a, b in zip(f, f[1:]))
    # the 1-layer count, term by term: forward 166 + sin/cos 12 + 2 x 20,
    # seed 11, adjoint 156 (the 1-layer adjoint keeps the forward's values)
    assert abs(bench.flops_per_eval(1, 21) - (218 + 11 + 156 + 15 / 21)) < 1e-9
    # the forward count is the gradient's forward sweep plus smearing and
    # likelihood terms, and below the fwd+grad count at every depth
    assert abs(bench.flops_per_eval_fwd(1, 21) - (166 + 2 + 19 / 21)) < 1e-9
    assert abs(bench.flops_per_eval_fwd(1, 21, table=True) - (218 + 2 + 19 / 21)) < 1e-9
    assert all(bench.flops_per_eval_fwd(n, 21) < bench.flops_per_eval(n, 21) for n in range(0, 21))


def test_peak_probe_library_builds_and_exports():
    from paper_2509_06924_gb300 import _build
    lib = ctypes.CDLL(_build.build_peak())
    assert lib.nr_peak_threads() == 256
    # bad arguments are refused before any device call
    ms, ops = ctypes.c_double(), ctypes.c_double()
    lib.nr_peak_run.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_void_p,
                                ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_double)]
    assert lib.nr_peak_run(7, 1, 1, 1, None, ctypes.byref(ms), ctypes.byref(ops)) == -1
    assert lib.nr_peak_run(0, 0, 1, 1, None, ctypes.byref(ms), ctypes.byref(ops)) == -1


def test_profile_record_reads_the_summary_format(tmp_path, monkeypatch):
    """The bench takes traffic and FP32 counts from a committed ncu summary
    only while its kernel-source hash matches; keys may contain a colon."""
    import bench
    (tmp_path / "profiles").mkdir()
    (tmp_path / "profiles" / "nr_mixed_grad_w.txt").write_text(
        "kernel: k<2, 1, 21>(A, B)\nkernel source sha256[:16]: abc\ndram bytes per full launch: 123\n"
        "fp32 lane ops per eval: 4.5\n\ncommand: ncu --a b: c\n")
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    monkeypatch.setattr(bench, "kernel_source_hash", lambda: "abc")
    rec = bench.profile_record("w")
    assert rec["dram bytes per full launch"] == "123" and rec["fp32 lane ops per eval"] == "4.5"
    assert rec["command"] == "ncu --a b: c"
    monkeypatch.setattr(bench, "kernel_source_hash", lambda: "other")
    assert bench.profile_record("w") == {}


def test_kernel_source_hash_ignores_comments_only(tmp_path, monkeypatch):
    import shutil

    import bench
    src = os.path.join(ROOT, "paper_2509_06924_gb300", "csrc")
    dst = tmp_path / "paper_2509_06924_gb300" / "csrc"
    dst.mkdir(parents=True)
    for f in bench.KERNEL_SOURCES:
        shutil.copy(os.path.join(src, f), dst / f)
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    h0 = bench.kernel_source_hash()
    p = dst / bench.KERNEL_SOURCES[-1]
    text = p.read_text()
    p.write_text("// a comment\n" + text.replace("\n", "  // trailing\n", 3))
    assert bench.kernel_source_hash() == h0
    p.write_text(text + "\nstatic int extra_symbol;\n")
    assert bench.kernel_source_hash() != h0


# ------------------------------------------------------- autotune cache ----
def test_tune_cache_round_trip(tmp_path):
    import json
    path = str(tmp_path / "tune.json")
    key1 = "NVIDIA GB300|152|2|21|12|17|t2"
    key2 = "NVIDIA GB300|152|0|17|1|13|t2"
    assert nr.tune_cache_get(path, key1) is None            # no file yet
    nr.tune_cache_put(path, key1, 1, 12, 4, 134.25)
    nr.tune_cache_put(path, key2, 0, 6, 7, 0.5)
    nr.tune_cache_put(path, key1, 1, 6, 3, 130.0)           # replaces the first entry
    assert nr.tune_cache_get(path, key1) == {"paired": 1, "tile_q": 6, "ctas_per_sm": 3, "ms": 130.0}
    assert nr.tune_cache_get(path, key2) == {"paired": 0, "tile_q": 6, "ctas_per_sm": 7, "ms": 0.5}
    assert nr.tune_cache_get(path, "absent|key") is None
    doc = json.load(open(path))                             # the file is plain JSON
    assert doc["version"] == 1 and set(doc["entries"]) == {key1, key2}
    assert doc["entries"][key2] == {"paired": 0, "tile_q": 6, "ctas_per_sm": 7, "ms": 0.5}


def test_tune_cache_tolerates_foreign_and_broken_files(tmp_path):
    import json
    path = tmp_path / "tune.json"
    # written by another tool: other field order, extra whitespace
    path.write_text(json.dumps({"entries": {"k": {"ms": 2.5, "ctas_per_sm": 2, "tile_q": 9, "paired": 0}},
                                "version": 1}, indent=3))
    assert nr.tune_cache_get(str(path), "k") == {"paired": 0, "tile_q": 9, "ctas_per_sm": 2, "ms": 2.5}
    path.write_text("{ not json")
    assert nr.tune_cache_get(str(path), "k") is None        # unreadable: an empty cache
    nr.tune_cache_put(str(path), "k2", 1, 3, 1)             # ... which a write replaces
    assert nr.tune_cache_get(str(path), "k2")["tile_q"] == 3
    with pytest.raises(nr.NRError):
        nr.tune_cache_put(str(path), 'bad"key', 1, 3, 1)


# --------------------------------------------- strong-scaling partition ----
def test_cost_partition_covers_every_stack_once_and_balances():
    from paper_2509_06924_gb300 import shard
    wl = W.make_workload("uneven", n_stacks=500)
    q_len = (wl.q_off[1:] - wl.q_off[:-1])[wl.dataset]
    cost = shard.stack_costs(wl.n_layers, q_len, wl.n_quad)
    for world in (1, 2, 3, 8):
        parts = shard.cost_partition(cost, world)
        allidx = np.sort(np.concatenate(parts))
        np.testing.assert_array_equal(allidx, np.arange(wl.n_stacks))
        loads = np.array([cost[p].sum() for p in parts])
        # LPT greedy: the largest load is within the largest single cost of the mean
        assert loads.max() <= loads.mean() + cost.max() + 1e-9
        assert all(np.all(np.diff(p) > 0) for p in parts)
