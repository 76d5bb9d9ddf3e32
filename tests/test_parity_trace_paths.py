"""GPU parity of every launch shape amc_check_trace may pick when it times
its candidates on the first call of a size class: the path by size with the
single-pass scan's stuck bitmap read through L1, from shared memory or not at
all, with and without tile groups; the reduce / carry / apply path forced at
any size; the epoch path forced on every trace longer than 2^21 ops (else the
single-pass scan alone).  AMC_TRACE_CANDIDATE picks one of them untimed.
Bit-exact against the oracle on every output, with and without initial
statuses; amc_check_trace_plan names the path each candidate takes."""
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


def check(amc, oracle_mod, ks, var, n_vars, init):
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


# (ops, variables, kind probabilities r / w / Push / Pull / Noop)
SHAPES = {
    "small_16": (4096, 16, None),
    "small_ragged": (40_003, 2048, [0.05, 0.5, 0.1, 0.1, 0.25]),
    "mid_64": (1 << 20, 64, [0.02, 0.6, 0.05, 0.05, 0.28]),
    "mid_4096": ((1 << 18) + 77, 4096, [0.05, 0.5, 0.1, 0.1, 0.25]),
    "wide_20000": ((1 << 20) + 5, 20_000, [0.05, 0.5, 0.1, 0.1, 0.25]),
    "long_wide": ((1 << 23) + 12_345, 40_000, [0.01, 0.6, 0.05, 0.05, 0.29]),
}
PATHS = {  # candidate -> path it takes for each shape (by size / forced)
    "small_16": ["small"] * 4 + ["small", "scan"],
    "small_ragged": ["small"] * 4 + ["small", "scan"],
    "mid_64": ["scan"] * 4 + ["warp_dense", "scan"],
    "mid_4096": ["warp_dense"] * 4 + ["warp_dense", "scan"],
    "wide_20000": ["scan"] * 4 + ["dense", "scan"],      # rows in global memory
    "long_wide": ["scan"] * 4 + ["dense", "epochs"],
}


@pytest.mark.parametrize("with_init", [False, True])
@pytest.mark.parametrize("cand", range(6))
@pytest.mark.parametrize("shape", sorted(SHAPES))
def test_candidate(amc, oracle_mod, monkeypatch, shape, cand, with_init):
    for k in ("AMC_SCAN_DENSE", "AMC_SCAN_TAIL", "AMC_SCAN_DENSE_SORT", "AMC_SCAN_FB_BITS", "AMC_SCAN_GROUP"):
        monkeypatch.delenv(k, raising=False)
    monkeypatch.setenv("AMC_TRACE_CANDIDATE", str(cand))
    n, nv, p = SHAPES[shape]
    rng = np.random.default_rng(900 + sorted(SHAPES).index(shape))
    ks, var = workloads.trace_random(rng, n, nv, **({} if p is None else {"p": p}))
    init = rng.integers(0, 5, nv).astype(np.uint8) if with_init else None
    assert amc.trace_plan(n, nv, with_init)[0] == PATHS[shape][cand]
    check(amc, oracle_mod, ks, var, nv, init)


def test_first_call_tunes_and_reports(amc, oracle_mod, monkeypatch):
    # without the override the first call of a size class times every
    # candidate; its outputs and those of the next call (the chosen one) match
    for k in ("AMC_TRACE_CANDIDATE", "AMC_AUTOTUNE"):
        monkeypatch.delenv(k, raising=False)
    rng = np.random.default_rng(950)
    n, nv = (1 << 19) + 3, 700
    ks, var = workloads.trace_random(rng, n, nv, p=[0.03, 0.5, 0.1, 0.1, 0.27])
    check(amc, oracle_mod, ks, var, nv, None)
    path, launches = amc.trace_plan(n, nv)
    assert path in amc.TRACE_PATHS and launches >= 1
    check(amc, oracle_mod, ks, var, nv, None)


@pytest.mark.parametrize("cand", [0, 1])
def test_guarded_check_candidates(amc, oracle_mod, monkeypatch, cand):
    # amc_check_guarded_trace times two candidates: the plain choice and both
    # passes on the reduce / carry / apply path, which over 20,000 variables
    # keeps its per-chunk rows in global memory
    monkeypatch.setenv("AMC_GUARDED_CANDIDATE", str(cand))
    w = workloads.vectorpu_calls(seed=95, n_arrays=10_000, space=1 << 20, n_calls=60_000, len_log2=(4.0, 10.0))
    exp = oracle_mod.vectorpu(**w)
    n = exp["kind_side"].size
    assert n >= 1 << 20
    A = w["arr_start"].size
    dev = torch.device("cuda")
    out = amc.check_trace(torch.from_numpy(exp["kind_side"]).to(dev), torch.from_numpy(exp["var"]).to(dev), 2 * A,
                          guarded=True)
    assert amc.sync_status() == 0
    assert np.array_equal(out["step_status"].cpu().numpy(), exp["step_status"])
    assert np.array_equal(out["final_status"].cpu().numpy(), exp["final_status"])
    assert np.array_equal(out["var_first_fault"].cpu().numpy(), exp["var_first_fault"])
    assert int(out["first_fault"].cpu()[0]) == exp["first_fault"]
