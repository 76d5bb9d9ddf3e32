"""amc_check_trace_noalloc, the allocation-free trace check, against the
oracle and against the workspace entry point amc_check_trace.

Some callers cannot allocate device memory themselves (their host owns every
allocation, they are plug-ins handed only inputs and outputs, or an allocation
would synchronise a latency-critical loop); this entry point takes its scratch
from a fixed array inside the library.  The test calls it through the C ABI
three times in a row -- a 2^22-op Zipf trace over 2^20 variables (both
limits), a 123,457-op trace with initial statuses that include F, and an
empty trace -- and checks every output against the oracle and against
amc_check_trace exactly (integer results: no tolerance).  It also checks that
sizes above the documented limits are rejected before any GPU work.  This file
is collected last so that a failure here does not hide any other test."""
import ctypes

import numpy as np
import pytest
import torch

import workloads

pytestmark = pytest.mark.gpu

AMC_E_RANGE = -2
MAX_OPS = 1 << 22
MAX_VARS = 1 << 20


@pytest.fixture(scope="module")
def amc():
    import paper_1910_11110_gb300 as m
    m.build()
    L = m.lib()
    P = ctypes.c_void_p
    L.amc_check_trace_noalloc.argtypes = [P, P, ctypes.c_int64, ctypes.c_int32, P, P, P, P, P, P]
    L.amc_check_trace_noalloc.restype = ctypes.c_int
    return m


def outputs(n_ops, n_vars, dev):
    return dict(step_status=torch.full((n_ops,), 0xEE, dtype=torch.uint8, device=dev),
                final_status=torch.full((n_vars,), 0xEE, dtype=torch.uint8, device=dev),
                var_first_fault=torch.full((n_vars,), -7, dtype=torch.int32, device=dev),
                first_fault=torch.full((1,), -7, dtype=torch.int64, device=dev))


def call_noalloc(amc, ks, var, n_vars, init, out):
    p = lambda t: None if t is None else ctypes.c_void_p(t.data_ptr())
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    return amc.lib().amc_check_trace_noalloc(p(ks), p(var), ks.numel(), n_vars, p(init), p(out["step_status"]),
                                            p(out["final_status"]), p(out["var_first_fault"]),
                                            p(out["first_fault"]), stream)


def test_noalloc_matches_oracle_and_workspace_entry_point(amc, oracle_mod):
    dev = torch.device("cuda")
    rng = np.random.default_rng(17)
    ks1, var1 = workloads.trace_zipf(MAX_OPS, MAX_VARS, seed=23, device=dev)
    ks2_h, var2_h = workloads.trace_random(rng, 123_457, 1000, kinds=(0, 1, 2, 3, 4, 5, 7))
    ks2, var2 = torch.from_numpy(ks2_h).to(dev), torch.from_numpy(var2_h).to(dev)
    init2_h = rng.integers(0, 5, 1000).astype(np.uint8)
    init2_h[:10] = 4                         # some variables stuck before the first op
    init2 = torch.from_numpy(init2_h).to(dev)
    init3 = torch.from_numpy(rng.integers(0, 5, 77).astype(np.uint8)).to(dev)
    empty_ks = torch.zeros(0, dtype=torch.uint8, device=dev)
    empty_var = torch.zeros(0, dtype=torch.int32, device=dev)
    cases = [(ks1, var1, MAX_VARS, None), (ks2, var2, 1000, init2), (empty_ks, empty_var, 77, init3)]
    for ks, var, nv, init in cases:          # three calls in a row, different shapes
        got = outputs(ks.numel(), nv, dev)
        assert call_noalloc(amc, ks, var, nv, init, got) == 0
        assert amc.sync_status() == 0
        exp = oracle_mod.check_trace(ks.cpu().numpy(), var.cpu().numpy(), nv,
                                     None if init is None else init.cpu().numpy())
        assert np.array_equal(got["step_status"].cpu().numpy(), exp[0])
        assert np.array_equal(got["final_status"].cpu().numpy(), exp[1])
        assert np.array_equal(got["var_first_fault"].cpu().numpy(), exp[2])
        assert int(got["first_fault"].cpu()[0]) == exp[3]
        if ks.numel() == 0:
            assert exp[3] == -1 and np.array_equal(exp[1], init.cpu().numpy())
            continue
        ref = amc.check_trace(ks, var, nv, init)
        assert amc.sync_status() == 0
        for k in ref:
            assert torch.equal(got[k], ref[k]), k


def test_noalloc_rejects_sizes_beyond_limits(amc):
    dev = torch.device("cuda")
    ks = torch.zeros(8, dtype=torch.uint8, device=dev)
    var = torch.zeros(8, dtype=torch.int32, device=dev)
    out = outputs(8, 4, dev)
    lib = amc.lib()
    p = lambda t: ctypes.c_void_p(t.data_ptr())
    s = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    args = (p(out["step_status"]), p(out["final_status"]), p(out["var_first_fault"]), p(out["first_fault"]), s)
    assert lib.amc_check_trace_noalloc(p(ks), p(var), MAX_OPS + 1, 4, None, *args) == AMC_E_RANGE
    assert lib.amc_check_trace_noalloc(p(ks), p(var), 8, MAX_VARS + 1, None, *args) == AMC_E_RANGE
    assert amc.sync_status() == 0
