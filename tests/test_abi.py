"""The C ABI library builds for sm_103a and exports every symbol that
include/*.h declares (no compute calls: runs without a GPU)."""
import ctypes
import glob
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        text = open(h).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        for m in re.finditer(r"\b(amc_\w+)\s*\(", text):
            names.add(m.group(1))
    return sorted(names)


@pytest.fixture(scope="module")
def libamc():
    import paper_1910_11110_gb300 as amc
    path = amc.build()
    return ctypes.CDLL(path)


def test_header_declares_entry_points():
    names = declared_functions()
    for n in ("amc_check_trace", "amc_check_guarded_trace", "amc_translate_vectorpu", "amc_check_batch",
              "amc_check_well_declared", "amc_check_trace_k",
              "amc_serve_submit", "amc_serve_poll", "amc_sync_status"):
        assert n in names


def test_library_exports_every_declared_symbol(libamc):
    missing = [n for n in declared_functions() if not hasattr(libamc, n)]
    assert not missing, missing


def test_error_strings(libamc):
    libamc.amc_error_string.restype = ctypes.c_char_p
    for code in range(0, -7, -1):
        assert libamc.amc_error_string(code)
    assert libamc.amc_version() >= 10000


def test_workspace_queries_are_sane(libamc):
    libamc.amc_check_trace_workspace.restype = ctypes.c_size_t
    libamc.amc_check_trace_workspace.argtypes = [ctypes.c_int64, ctypes.c_int32]
    a = libamc.amc_check_trace_workspace(1 << 20, 1 << 10)
    b = libamc.amc_check_trace_workspace(1 << 21, 1 << 10)
    assert 0 < a < b
    assert libamc.amc_check_trace_workspace(-1, 4) == 0


def test_binding_fails_loudly_without_library(monkeypatch, tmp_path):
    import paper_1910_11110_gb300 as amc
    monkeypatch.setattr(amc, "LIB_PATH", str(tmp_path / "missing.so"))
    monkeypatch.setattr(amc, "_lib", None)
    with pytest.raises(RuntimeError):
        amc.lib()


def test_workspace_sizes_at_the_bench_size(libamc):
    # the trace check's scratch stays about 5.5 B per op at 2^30 ops over 2^20
    # variables (the epoch path shares one region with its fallback); the
    # host-buffer check's device scratch is three chunk slots (6 B per op) plus
    # one chunk's scan (with the dense prefix's rows), whatever the trace length
    libamc.amc_check_trace_workspace.restype = ctypes.c_size_t
    libamc.amc_check_trace_workspace.argtypes = [ctypes.c_int64, ctypes.c_int32]
    libamc.amc_check_trace_host_workspace.restype = ctypes.c_size_t
    libamc.amc_check_trace_host_workspace.argtypes = [ctypes.c_int64, ctypes.c_int32, ctypes.c_int64]
    n, v = 1 << 30, 1 << 20
    ws = libamc.amc_check_trace_workspace(n, v)
    assert 5 * n < ws < 6 * n
    h = libamc.amc_check_trace_host_workspace(n, v, 0)
    h2 = libamc.amc_check_trace_host_workspace(n // 4, v, 0)
    assert h == h2                      # independent of the trace length
    assert 18 * (1 << 25) < h < 48 * (1 << 25)
    assert libamc.amc_check_trace_host_workspace(n, v, 1 << 20) < h
    assert libamc.amc_check_trace_host_workspace(-1, v, 0) == 0


def test_epoch_shape_follows_its_override(libamc, monkeypatch):
    # the long-trace path's shape (first part, epochs) is host logic read per
    # call: the workspace query follows AMC_SCAN_TAIL without a GPU (the query
    # is the larger of the single-pass and the epoch path's needs)
    libamc.amc_check_trace_workspace.restype = ctypes.c_size_t
    libamc.amc_check_trace_workspace.argtypes = [ctypes.c_int64, ctypes.c_int32]
    ws = libamc.amc_check_trace_workspace
    # (below 2^20 ops, where the global-row reduce / carry / apply scratch that
    # a tuner candidate may take is not part of the query)
    n, v = 3 << 18, 1 << 20
    monkeypatch.delenv("AMC_SCAN_TAIL", raising=False)
    plain, few = ws(n, v), ws(n, 16_384)     # below 2^29 ops: no epoch path
    monkeypatch.setenv("AMC_SCAN_TAIL", "16,-2")
    assert ws(n, v) > plain                  # forced: pairs for 2^16 ops, slots for epochs to 3 * 2^18
    assert ws(n, 16_384) == few              # too few variables: the path is not taken
    monkeypatch.setenv("AMC_SCAN_TAIL", "0")
    assert ws(n, v) == plain                 # "0" switches the path off
    monkeypatch.setenv("AMC_SCAN_TAIL", "30,-2")
    assert ws(n, v) == plain                 # a first part beyond 2^27 ops is not accepted
    monkeypatch.setenv("AMC_SCAN_TAIL", "16,-7")
    assert ws(n, v) == plain                 # nor a growth beyond 2^4


def test_trace_plan_follows_the_size_rule(monkeypatch):
    # host logic only: which path a check of these sizes takes before any
    # timing, and the kernels it launches
    import paper_1910_11110_gb300 as amc
    for k in ("AMC_SCAN_DENSE", "AMC_SCAN_TAIL", "AMC_SCAN_DENSE_SORT"):
        monkeypatch.delenv(k, raising=False)
    plan = amc.trace_plan
    assert plan(4096, 16) == ("small", 1)
    assert plan(1 << 16, 2048) == ("small", 1)
    assert plan(1 << 16, 2048, has_init=True) == ("small", 1)
    assert plan((1 << 16) + 1, 16)[0] == "scan"           # 16 variables: the scan at every length
    assert plan(1 << 16, 4096) == ("warp_dense", 5)       # 2^12 variables from 2^15 ops
    assert plan(1 << 14, 4096)[0] == "scan"
    assert plan(1 << 21, 512) == ("warp_dense", 5)        # 2^9 variables from 2^21 ops
    assert plan(1 << 20, 512)[0] == "scan"
    assert plan(1 << 11, 16384) == ("dense", 3)           # 2^14 variables from 2^11 ops
    assert plan(1 << 24, 1 << 20) == ("prefix", 7)
    assert plan(1 << 24, 1 << 20, has_init=True)[0] == "scan"
    # the epoch path from 2^29 ops: pairs + 3 radix passes (3 kernels each) +
    # segmented scan (reduce, carry, apply) + bitmap, then 12 kernels per epoch
    # (filter, block sums, offsets, gather, one radix pass, bucket check,
    # gated fallback and merge; 2^21 -> 2^23 -> 2^25 -> 2^27 -> 2^29 -> 2^30)
    assert plan(1 << 30, 1 << 20) == ("epochs", 14 + 12 * 5)
    assert plan(1 << 29, 1 << 20) == ("epochs", 14 + 12 * 4)
    # the epoch path's bounds: from 2^29 ops, 16,385 to 2^20 variables (the
    # stuck bitmap fills 128 KB of shared memory; fewer variables take the
    # reduce / carry / apply path)
    assert plan(1 << 29, 16_385) == ("epochs", 14 + 12 * 4)
    assert plan((1 << 29) - 1, 16_385)[0] == "prefix"
    assert plan(1 << 29, 16_384)[0] == "dense"
    assert plan(1 << 29, (1 << 20) + 1)[0] == "scan"
    monkeypatch.setenv("AMC_SCAN_TAIL", "0")
    assert plan(1 << 30, 1 << 20) == ("prefix", 7)
    monkeypatch.setenv("AMC_SCAN_DENSE", "0")
    assert plan(1 << 16, 4096) == ("scan", 2)
    monkeypatch.setenv("AMC_SCAN_DENSE", "1")
    assert plan(1 << 20, 64) == ("warp_dense", 5)
    monkeypatch.setenv("AMC_SCAN_DENSE_SORT", "1")
    assert plan(1 << 20, 64) == ("dense", 3)
    with pytest.raises(RuntimeError):
        plan(-1, 16)
