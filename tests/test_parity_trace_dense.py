"""GPU parity of the reduce / carry / apply path of the trace check.

Traces over at most 16,384 variables take that path from 2^20 ops on (up to
8,192 variables as warp-sequential batches, above that with tile sorts);
AMC_SCAN_DENSE=1 forces it at any size and AMC_SCAN_DENSE_SORT=1 the sorted
variant, so that ragged tails, single tiles, chunks of several tiles (more
than 2,048 tiles), one variable, the largest variable count, initial
statuses and the guard pass all run through both.
Bit-exact against the oracle on every output."""
import numpy as np
import pytest
import torch

import workloads

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def amc():
    import paper_1910_11110_gb300 as m
    m.build()
    return m


def check(amc, oracle_mod, ks, var, n_vars, init=None):
    exp = oracle_mod.check_trace(ks, var, n_vars, init)
    dev = torch.device("cuda")
    out = amc.check_trace(torch.from_numpy(ks).to(dev), torch.from_numpy(var).to(dev), n_vars,
                          None if init is None else torch.from_numpy(init).to(dev))
    assert amc.sync_status() == 0
    got = (out["step_status"].cpu().numpy(), out["final_status"].cpu().numpy(),
           out["var_first_fault"].cpu().numpy(), int(out["first_fault"].cpu()[0]))
    for e, g in zip(exp[:3], got[:3]):
        assert np.array_equal(e, g), np.nonzero(e != g)[0][:10]
    assert exp[3] == got[3]


CASES = {
    "one_op": lambda rng: (workloads.trace_random(rng, 1, 1), 1, None),
    "ragged_small": lambda rng: (workloads.trace_random(rng, 3 * 4096 + 17, 5), 5, None),
    "one_variable": lambda rng: (workloads.trace_random(rng, 70_001, 1, p=[0.0, 0.5, 0.0, 0.0, 0.5]), 1, None),
    "low_fault": lambda rng: (workloads.trace_random(rng, 400_003, 300, p=[0.02, 0.6, 0.05, 0.05, 0.28]), 300, None),
    "max_vars": lambda rng: (workloads.trace_random(rng, 300_000, 16384, p=[0.05, 0.5, 0.1, 0.1, 0.25]), 16384, None),
    "multi_tile_chunks": lambda rng: (workloads.trace_random(rng, 2100 * 4096 + 123, 4096,
                                                             p=[0.03, 0.5, 0.1, 0.1, 0.27]), 4096, None),
    "zipf": lambda rng: (workloads.trace_random(rng, 500_000, 8192, zipf_s=1.05), 8192, None),
}


@pytest.mark.parametrize("variant", ["warp", "sort"])
@pytest.mark.parametrize("case", sorted(CASES))
def test_dense_path(amc, oracle_mod, monkeypatch, case, variant):
    # up to 8,192 variables warp-sequential batches by default; "sort" forces the tile sorts
    monkeypatch.setenv("AMC_SCAN_DENSE", "1")
    monkeypatch.setenv("AMC_SCAN_DENSE_SORT", "1" if variant == "sort" else "0")
    rng = np.random.default_rng(41 + sorted(CASES).index(case))
    (ks, var), n_vars, init = CASES[case](rng)
    check(amc, oracle_mod, ks, var, n_vars, init)


def test_dense_path_initial_statuses(amc, oracle_mod, monkeypatch):
    monkeypatch.setenv("AMC_SCAN_DENSE", "1")
    rng = np.random.default_rng(49)
    ks, var = workloads.trace_random(rng, 90_000, 64)
    init = rng.integers(0, 5, 64).astype(np.uint8)
    check(amc, oracle_mod, ks, var, 64, init)


@pytest.mark.parametrize("dense", ["1", "0"])
def test_dense_and_list_paths_agree_at_default_threshold(amc, oracle_mod, monkeypatch, dense):
    # 2^20 ops over 2,000 variables: the dense path by default, the list path when disabled
    monkeypatch.setenv("AMC_SCAN_DENSE", dense)
    rng = np.random.default_rng(50)
    ks, var = workloads.trace_random(rng, 1 << 20, 2000, p=[0.03, 0.5, 0.1, 0.1, 0.27])
    check(amc, oracle_mod, ks, var, 2000)


@pytest.mark.parametrize("variant", ["warp", "sort"])
def test_dense_path_guarded(amc, oracle_mod, monkeypatch, variant):
    monkeypatch.setenv("AMC_SCAN_DENSE", "1")
    monkeypatch.setenv("AMC_SCAN_DENSE_SORT", "1" if variant == "sort" else "0")
    w = workloads.vectorpu_calls(seed=51, n_arrays=64, space=1 << 14, n_calls=20_000,
                                 len_log2=(4.0, 10.0), drop_p=0.01)
    res = oracle_mod.vectorpu(**w)
    A = len(w["arr_start"])
    dev = torch.device("cuda")
    out = amc.check_trace(torch.from_numpy(res["kind_side"]).to(dev), torch.from_numpy(res["var"]).to(dev),
                          2 * A, guarded=True)
    assert amc.sync_status() == 0
    assert np.array_equal(out["step_status"].cpu().numpy(), res["step_status"])
    assert np.array_equal(out["final_status"].cpu().numpy(), res["final_status"])
    assert np.array_equal(out["var_first_fault"].cpu().numpy(), res["var_first_fault"])
    assert int(out["first_fault"].cpu()[0]) == res["first_fault"]


def test_dense_path_reports_bad_input(amc, monkeypatch):
    monkeypatch.setenv("AMC_SCAN_DENSE", "1")
    dev = torch.device("cuda")
    ks = torch.tensor([0, 1, 2], dtype=torch.uint8, device=dev)
    var = torch.tensor([0, 5, 1], dtype=torch.int32, device=dev)
    amc.check_trace(ks, var, 4)
    assert amc.sync_status() == amc.E_RANGE
    ks = torch.tensor([0, 0x21, 2], dtype=torch.uint8, device=dev)
    var = torch.tensor([0, 1, 1], dtype=torch.int32, device=dev)
    amc.check_trace(ks, var, 4)
    assert amc.sync_status() == amc.E_INVALID
    assert amc.sync_status() == 0


# ---- prefix split: traces over more than 16,384 variables ------------------
# From 2^24 ops the first 2^22 ops take the reduce / carry / apply path with
# per-chunk rows in global memory and the rest the single-pass kernel from the
# prefix's final statuses; AMC_SCAN_PREFIX=k forces a 2^k-op prefix at any size.

def test_prefix_split_zipf(amc, oracle_mod, monkeypatch):
    monkeypatch.setenv("AMC_SCAN_PREFIX", "18")
    ks, var = workloads.trace_zipf(3 * (1 << 20) + 5, 1 << 20, seed=52, device="cuda")
    check(amc, oracle_mod, ks.cpu().numpy(), var.cpu().numpy(), 1 << 20)


def test_prefix_split_ragged(amc, oracle_mod, monkeypatch):
    monkeypatch.setenv("AMC_SCAN_PREFIX", "14")
    rng = np.random.default_rng(53)
    ks, var = workloads.trace_random(rng, 200_003, 70_000, zipf_s=1.05)
    check(amc, oracle_mod, ks, var, 70_000)


def test_prefix_split_initial_statuses(amc, oracle_mod, monkeypatch):
    monkeypatch.setenv("AMC_SCAN_PREFIX", "15")
    rng = np.random.default_rng(54)
    ks, var = workloads.trace_random(rng, 150_000, 20_000)
    init = rng.integers(0, 5, 20_000).astype(np.uint8)
    check(amc, oracle_mod, ks, var, 20_000, init)


def test_prefix_split_guarded_gt_at_boundary(amc, oracle_mod, monkeypatch):
    # 9,000 arrays (18,000 variables); this seed's translated trace has a GT at
    # position 2^15 - 1, so the GT / EN pair straddles a 2^15-op prefix
    monkeypatch.setenv("AMC_SCAN_PREFIX", "15")
    w = workloads.vectorpu_calls(seed=61, n_arrays=9000, space=1 << 16, n_calls=30_000,
                                 len_log2=(4.0, 9.0), drop_p=0.01)
    res = oracle_mod.vectorpu(**w)
    assert (res["kind_side"][(1 << 15) - 1] & 15) == 6
    A = len(w["arr_start"])
    dev = torch.device("cuda")
    out = amc.check_trace(torch.from_numpy(res["kind_side"]).to(dev), torch.from_numpy(res["var"]).to(dev),
                          2 * A, guarded=True)
    assert amc.sync_status() == 0
    assert np.array_equal(out["step_status"].cpu().numpy(), res["step_status"])
    assert np.array_equal(out["final_status"].cpu().numpy(), res["final_status"])
    assert np.array_equal(out["var_first_fault"].cpu().numpy(), res["var_first_fault"])
    assert int(out["first_fault"].cpu()[0]) == res["first_fault"]
