"""GPU parity of the trace check over k memory locations (amc_check_trace_k)
against the oracle, bit-exact on every output: k = 1..7, traces spanning many
sort tiles with ragged tails, runs of one variable across tiles, initial
statuses including stuck ones, the two-location embedding against the
two-location GPU check, a 2^24-op trace, the empty trace and bad input."""
import numpy as np
import pytest
import torch

import workloads

pytestmark = pytest.mark.gpu
KL_F = 0x80


@pytest.fixture(scope="module")
def amc():
    import paper_1910_11110_gb300 as m
    m.build()
    return m


def random_kloc(rng, n, n_vars, k, zipf=False):
    kind = rng.choice(4, size=n, p=[0.4, 0.2, 0.3, 0.1])
    a = rng.integers(0, k, n)
    b = (a + rng.integers(1, k, n)) % k if k > 1 else a
    op = np.where(kind == 3, 3, np.where(kind == 2, kind | a << 2 | b << 5, kind | a << 2)).astype(np.uint8)
    if k == 1:
        op[kind == 2] = 3
    if zipf:
        var = np.minimum(np.searchsorted(workloads.zipf_cdf(n_vars), rng.random(n)), n_vars - 1)
    else:
        var = rng.integers(0, n_vars, n)
    return op, var.astype(np.int32)


def check(amc, oracle_mod, op, var, n_vars, k, init=None):
    exp = oracle_mod.check_trace_k(op, var, n_vars, k, init)
    t = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()
    out = amc.check_trace_k(t(op), t(var), n_vars, k, None if init is None else t(init))
    assert amc.sync_status() == 0
    got = (out["step_status"].cpu().numpy(), out["final_status"].cpu().numpy(),
           out["var_first_fault"].cpu().numpy(), int(out["first_fault"].cpu()[0]))
    for name, e, g in zip(("step_status", "final_status", "var_first_fault"), exp[:3], got[:3]):
        assert np.array_equal(e, g), (name, np.nonzero(e != g)[0][:10])
    assert exp[3] == got[3]


@pytest.mark.parametrize("k", [1, 2, 3, 4, 5, 6, 7])
def test_random_traces(amc, oracle_mod, k):
    rng = np.random.default_rng(300 + k)
    op, var = random_kloc(rng, 50_001, 3_000, k, zipf=True)
    init = rng.integers(1, 1 << k, 3_000).astype(np.uint8)
    init[:50] = KL_F
    check(amc, oracle_mod, op, var, 3_000, k)
    check(amc, oracle_mod, op, var, 3_000, k, init)


def test_long_runs_across_tiles(amc, oracle_mod):
    # a few variables, reads and copies that rarely fault: runs of thousands of
    # ops per variable cross many 2,048-pair tiles (the carry between tiles)
    rng = np.random.default_rng(310)
    k, n = 4, 300_003
    op = np.full(n, 3, np.uint8)
    var = rng.integers(0, 5, n).astype(np.int32)
    pick = rng.random(n)
    op[pick < 0.5] = 0 | 0 << 2                                  # r at 0
    op[(pick >= 0.5) & (pick < 0.7)] = 2 | 0 << 2 | 2 << 5       # copy 0 -> 2
    op[(pick >= 0.7) & (pick < 0.72)] = 1 | 0 << 2               # w at 0
    op[-1000:] = 0 | 3 << 2                                      # r at 3: faults at the end
    check(amc, oracle_mod, op, var, 5, k)


def test_two_location_embedding(amc, oracle_mod):
    # k = 2 on the embedded two-location trace equals the two-location check
    rng = np.random.default_rng(311)
    ks, var = workloads.trace_random(rng, 100_000, 2_000, zipf_s=1.05)
    kind, side = ks & 15, ks >> 4
    op = np.select([kind == 0, kind == 1, kind == 2, kind == 3],
                   [0 | side << 2, 1 | side << 2, 2 | side << 2 | (1 - side) << 5, 2 | (1 - side) << 2 | side << 5],
                   3).astype(np.uint8)
    t = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()
    a = amc.check_trace_k(t(op), t(var), 2_000, 2)
    b = amc.check_trace(t(ks), t(var), 2_000)
    assert amc.sync_status() == 0
    m = lambda s: torch.where(s == KL_F, torch.full_like(s, 4), s)
    assert torch.equal(m(a["step_status"]), b["step_status"])
    assert torch.equal(m(a["final_status"]), b["final_status"])
    assert torch.equal(a["var_first_fault"], b["var_first_fault"])
    assert torch.equal(a["first_fault"], b["first_fault"])


def test_large(amc, oracle_mod):
    rng = np.random.default_rng(312)
    op, var = random_kloc(rng, 1 << 24, 1 << 16, 5, zipf=True)
    check(amc, oracle_mod, op, var, 1 << 16, 5)


def test_empty_and_bad_input(amc, oracle_mod):
    check(amc, oracle_mod, np.zeros(0, np.uint8), np.zeros(0, np.int32), 10, 3,
          np.arange(10, dtype=np.uint8) % 7 + 1)
    t = lambda a: torch.from_numpy(np.asarray(a)).cuda()
    amc.check_trace_k(t(np.array([2 | 1 << 2 | 1 << 5], np.uint8)), t(np.array([0], np.int32)), 4, 3)
    assert amc.sync_status() == amc.E_INVALID                    # copy 1 -> 1
    amc.check_trace_k(t(np.array([0 | 3 << 2], np.uint8)), t(np.array([0], np.int32)), 4, 3)
    assert amc.sync_status() == amc.E_INVALID                    # location 3 with k = 3
    amc.check_trace_k(t(np.array([0], np.uint8)), t(np.array([9], np.int32)), 4, 3)
    assert amc.sync_status() == amc.E_RANGE
    amc.check_trace_k(t(np.array([0], np.uint8)), t(np.array([0], np.int32)), 4, 3,
                      t(np.array([1, 8, 1, 1], np.uint8)))
    assert amc.sync_status() == amc.E_INVALID                    # initial status with location 3 valid
    with pytest.raises(amc.AmcError):
        amc.check_trace_k(t(np.array([0], np.uint8)), t(np.array([0], np.int32)), 4, 8)
    assert amc.sync_status() == 0
