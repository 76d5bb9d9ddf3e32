"""GPU parity of amc_check_trace_host (the trace check over host buffers, cut
into chunks that are copied in, checked and copied out in a pipeline) with the
oracle, element by element.

Section 3.2 fixes every status after every op; the chunked check must give
exactly the outputs of one check over the whole trace, so the cases put faults
on both sides of chunk boundaries, run more chunks than device slots, give
initial statuses, mix the few-variable and many-variable paths and use
pageable as well as pinned host buffers."""
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


def host(a, pinned=True):
    t = torch.from_numpy(np.ascontiguousarray(a))
    return t.pin_memory() if pinned else t.clone()


def check(amc, oracle_mod, ks, var, n_vars, init=None, chunk_ops=0, pinned=True):
    exp = oracle_mod.check_trace(ks, var, n_vars, init)
    out = amc.check_trace_host(host(ks, pinned), host(var, pinned), n_vars,
                               None if init is None else host(init, pinned), chunk_ops=chunk_ops)
    assert amc.sync_status() == 0
    got = (out["step_status"].numpy(), out["final_status"].numpy(), out["var_first_fault"].numpy(),
           int(out["first_fault"][0]))
    for name, e, g in zip(("step_status", "final_status", "var_first_fault"), exp[:3], got[:3]):
        assert np.array_equal(e, g), (name, np.nonzero(e != g)[0][:10])
    assert exp[3] == got[3]


CASES = {
    # (n_ops, n_vars, kind mix or None, zipf exponent or None, chunk_ops)
    "ragged_many_chunks": (7 * 4096 + 123, 50, [0.03, 0.5, 0.1, 0.1, 0.27], None, 4096),
    "one_chunk": (10_000, 1000, None, None, 0),
    "chunk_not_multiple_of_tile": (100_000, 3000, None, 1.05, 5000),
    "zipf_many_vars": (3 * (1 << 20) + 5, 1 << 20, None, 1.05, 1 << 18),
    "few_vars_dense_chunks": ((1 << 21) + 17, 300, [0.01, 0.6, 0.05, 0.05, 0.29], None, 1 << 20),
}


@pytest.mark.parametrize("case", sorted(CASES))
def test_chunked_host_check(amc, oracle_mod, case):
    n, n_vars, p, zipf_s, chunk = CASES[case]
    rng = np.random.default_rng(71 + sorted(CASES).index(case))
    kw = {}
    if p is not None:
        kw["p"] = p
    if zipf_s is not None:
        kw["zipf_s"] = zipf_s
    ks, var = workloads.trace_random(rng, n, n_vars, **kw)
    check(amc, oracle_mod, ks, var, n_vars, chunk_ops=chunk)


def test_initial_statuses(amc, oracle_mod):
    rng = np.random.default_rng(80)
    ks, var = workloads.trace_random(rng, 40_000, 2000)
    init = rng.integers(0, 5, 2000).astype(np.uint8)
    check(amc, oracle_mod, ks, var, 2000, init, chunk_ops=8192)


def test_pageable_buffers(amc, oracle_mod):
    rng = np.random.default_rng(81)
    ks, var = workloads.trace_random(rng, 30_000, 700)
    check(amc, oracle_mod, ks, var, 700, chunk_ops=4096, pinned=False)


def test_faults_on_chunk_boundaries(amc, oracle_mod):
    # 4,096-op chunks; variable 1 faults at the last op of chunk 0, variable 0
    # at the first op of chunk 1, variable 2 faults in chunk 0 and is accessed
    # again in every later chunk (F stays, its first fault stays in chunk 0)
    C = 4096
    n = 4 * C
    ks = np.full(n, 4, np.uint8)              # Noop on the CPU side
    var = np.full(n, 3, np.int32)
    ks[C - 1], var[C - 1] = 0x10, 1           # GPU read of a CPU-only variable: F
    ks[C], var[C] = 0x10, 0
    ks[100], var[100] = 0x10, 2
    for j in (C + 5, 2 * C, 3 * C + 9):
        ks[j], var[j] = 0x01, 2               # CPU write to an F variable
    check(amc, oracle_mod, ks, var, 4, chunk_ops=C)


def test_empty_trace(amc, oracle_mod):
    ks = np.zeros(0, np.uint8)
    var = np.zeros(0, np.int32)
    check(amc, oracle_mod, ks, var, 5)
    check(amc, oracle_mod, ks, var, 5, np.array([0, 1, 2, 3, 4], np.uint8))


def test_default_chunks_with_prefix_split(amc, oracle_mod):
    # 2^25 + 4,099 ops over 2^20 variables: two default chunks, the first
    # large enough for the dense prefix, the second from its final statuses
    ks, var = workloads.trace_zipf((1 << 25) + 4099, 1 << 20, seed=82, device="cpu")
    check(amc, oracle_mod, ks.numpy(), var.numpy(), 1 << 20)


def test_matches_device_check(amc):
    # the same trace through amc_check_trace on device buffers
    rng = np.random.default_rng(83)
    ks, var = workloads.trace_random(rng, 200_000, 10_000, zipf_s=1.05)
    dev = torch.device("cuda")
    d = amc.check_trace(torch.from_numpy(ks).to(dev), torch.from_numpy(var).to(dev), 10_000)
    h = amc.check_trace_host(host(ks), host(var), 10_000, chunk_ops=16384)
    assert amc.sync_status() == 0
    for k in ("step_status", "final_status", "var_first_fault", "first_fault"):
        assert torch.equal(d[k].cpu(), h[k]), k


def test_reports_bad_ids(amc):
    ks = np.zeros(3 * 4096, np.uint8)
    var = np.zeros(3 * 4096, np.int32)
    var[2 * 4096 + 7] = 9                     # out of range, in the third chunk
    amc.check_trace_host(host(ks), host(var), 4, chunk_ops=4096)
    assert amc.sync_status() == amc.E_RANGE
    assert amc.sync_status() == 0


def test_workspace_too_small(amc):
    ks = host(np.zeros(5000, np.uint8))
    var = host(np.zeros(5000, np.int32))
    need = amc.trace_host_workspace_bytes(5000, 4, 4096)
    ws = torch.empty(need + 256, dtype=torch.uint8, device="cuda")
    ws = ws[(-ws.data_ptr()) % 256:][:need - 256]
    with pytest.raises(amc.AmcError):
        amc.check_trace_host(ks, var, 4, chunk_ops=4096, workspace=ws)
