"""GPU parity of the trace check when CTAs take several tiles per claim.

The group path streams G consecutive tiles, compacts their live ops (ops on
variables not yet known to be stuck) and handles them together; a group with
more live ops than one tile's buffers falls back to the tile path tile by
tile.  AMC_SCAN_GROUP=-N forces every claim to take N tiles (so both the group
path and its fallback run on every trace shape); AMC_SCAN_GROUP=N caps the
adaptive choice at N.  Bit-exact against the oracle on every output."""
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


def case_random_ragged():
    rng = np.random.default_rng(31)
    ks, var = workloads.trace_random(rng, 21 * 4096 + 17, 5)
    return ks, var, 5, None


def case_zipf_many_tiles():
    ks, var = workloads.trace_zipf(1 << 22, 1 << 16, seed=32, device="cuda")
    return ks.cpu().numpy(), var.cpu().numpy(), 1 << 16, None


def case_zipf_wide_ids():
    # 2^21 variables: 64-bit sort keys
    ks, var = workloads.trace_zipf(3 * (1 << 20) + 5, 1 << 21, seed=33, device="cuda")
    return ks.cpu().numpy(), var.cpu().numpy(), 1 << 21, None


def case_one_variable():
    rng = np.random.default_rng(34)
    ks, var = workloads.trace_random(rng, 40 * 4096 + 3, 1, p=[0.0, 0.5, 0.0, 0.0, 0.5])
    return ks, var, 1, None


def case_low_fault():
    rng = np.random.default_rng(35)
    ks, var = workloads.trace_random(rng, 300_000, 5000, p=[0.02, 0.6, 0.05, 0.05, 0.28])
    return ks, var, 5000, None


def case_initial_statuses():
    rng = np.random.default_rng(36)
    ks, var = workloads.trace_random(rng, 90_000, 64)
    init = rng.integers(0, 5, 64).astype(np.uint8)
    return ks, var, 64, init


CASES = {"random_ragged": case_random_ragged, "zipf_many_tiles": case_zipf_many_tiles,
         "zipf_wide_ids": case_zipf_wide_ids, "one_variable": case_one_variable,
         "low_fault": case_low_fault, "initial_statuses": case_initial_statuses}


@pytest.mark.parametrize("group", ["-2", "-3", "-16", "16"])
@pytest.mark.parametrize("case", sorted(CASES))
def test_group_path(amc, oracle_mod, monkeypatch, group, case):
    monkeypatch.setenv("AMC_SCAN_GROUP", group)
    ks, var, n_vars, init = CASES[case]()
    check(amc, oracle_mod, ks, var, n_vars, init)


@pytest.mark.parametrize("group", ["-4", "-16"])
def test_group_path_guarded(amc, oracle_mod, monkeypatch, group):
    monkeypatch.setenv("AMC_SCAN_GROUP", group)
    w = workloads.vectorpu_calls(seed=37, n_arrays=64, space=1 << 14, n_calls=20_000,
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
