"""GPU parity of the epoch path for long traces (the first part checked by
sorting its ops by variable, then per epoch: stream filter on the stuck bitmap,
the compacted candidates checked by sorting them by variable from the epoch's
start statuses, which also adds the variables that become stuck to the
bitmap).

Traces over 16,385 to 2^20 variables take it from 2^29 ops on (first part 2^21
ops, each epoch ending at four times its start); AMC_SCAN_TAIL="s,e" forces a
first part of 2^s ops and epochs of 2^e ops, "s,-g" epochs ending at 2^g times
their start, at any length, so that many epochs, ragged last epochs, epochs
with almost every op a candidate, runs of one variable across many sort tiles,
initial statuses and bad input all run.  Bit-exact against the oracle on every
output."""
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
    for name, e, g in zip(("step_status", "final_status", "var_first_fault"), exp[:3], got[:3]):
        assert np.array_equal(e, g), (name, np.nonzero(e != g)[0][:10])
    assert exp[3] == got[3]


@pytest.mark.parametrize("shape", ["18,18", "16,20", "20,16"])
def test_zipf_epochs(amc, oracle_mod, monkeypatch, shape):
    monkeypatch.setenv("AMC_SCAN_TAIL", shape)
    ks, var = workloads.trace_zipf(3 * (1 << 20) + 5, 1 << 20, seed=90, device="cuda")
    check(amc, oracle_mod, ks.cpu().numpy(), var.cpu().numpy(), 1 << 20)


def test_initial_statuses(amc, oracle_mod, monkeypatch):
    monkeypatch.setenv("AMC_SCAN_TAIL", "14,14")
    rng = np.random.default_rng(91)
    ks, var = workloads.trace_random(rng, 300_007, 40_000, zipf_s=1.05)
    init = rng.integers(0, 5, 40_000).astype(np.uint8)
    check(amc, oracle_mod, ks, var, 40_000, init)


def test_every_op_a_candidate(amc, oracle_mod, monkeypatch):
    # writes and Noops only: nothing faults, every op of every epoch is checked
    monkeypatch.setenv("AMC_SCAN_TAIL", "15,15")
    rng = np.random.default_rng(92)
    ks, var = workloads.trace_random(rng, 200_003, 20_000, p=[0.0, 0.7, 0.0, 0.0, 0.3])
    check(amc, oracle_mod, ks, var, 20_000)


def test_faults_late_and_uniform_ids(amc, oracle_mod, monkeypatch):
    monkeypatch.setenv("AMC_SCAN_TAIL", "13,14")
    rng = np.random.default_rng(93)
    ks, var = workloads.trace_random(rng, 150_001, 17_000, p=[0.01, 0.6, 0.04, 0.04, 0.31])
    check(amc, oracle_mod, ks, var, 17_000)


def test_bad_input_in_the_tail(amc, monkeypatch):
    monkeypatch.setenv("AMC_SCAN_TAIL", "13,13")
    dev = torch.device("cuda")
    n, nv = 50_000, 20_000
    ks = torch.zeros(n, dtype=torch.uint8, device=dev)
    var = torch.arange(n, dtype=torch.int32, device=dev) % nv
    var[40_000] = nv + 3                           # id out of range, in an epoch
    amc.check_trace(ks, var, nv)
    assert amc.sync_status() == amc.E_RANGE
    var[40_000] = 5
    ks[30_001] = 0x21                              # malformed byte
    amc.check_trace(ks, var, nv)
    assert amc.sync_status() == amc.E_INVALID
    ks[30_001] = 6                                 # GT in a plain check
    amc.check_trace(ks, var, nv)
    assert amc.sync_status() == amc.E_INVALID
    assert amc.sync_status() == 0


def test_default_split_at_2p29(amc, oracle_mod):
    # 2^29 ops over 2^20 variables: the default first part (2^21 ops) and
    # epochs ending at 2^23, 2^25, 2^27 and 2^29 ops, against the oracle on
    # every output
    ks, var = workloads.trace_zipf(1 << 29, 1 << 20, seed=94, device="cuda")
    check(amc, oracle_mod, ks.cpu().numpy(), var.cpu().numpy(), 1 << 20)


def test_overflow_falls_back_in_one_epoch(amc, oracle_mod, monkeypatch):
    # epochs of 2^16 ops after a 2^15-op first part; the third epoch holds a
    # burst of writes on variables never touched before (none faults there),
    # more candidates than its chunks' slots: that epoch is rechecked whole,
    # the others take the compacted candidates
    monkeypatch.setenv("AMC_SCAN_TAIL", "15,16")
    rng = np.random.default_rng(95)
    nv = 30_000
    ks, var = workloads.trace_random(rng, 300_000, 20_000, zipf_s=1.05)
    lo = (1 << 15) + 2 * (1 << 16) + 1000
    ks[lo:lo + 9000] = 0x01                          # CPU writes
    var[lo:lo + 9000] = 20_000 + (np.arange(9000) % 10_000)
    check(amc, oracle_mod, ks, var, nv)


@pytest.mark.parametrize("shape", ["14,-2", "13,-1", "16,-3"])
def test_zipf_growing_epochs(amc, oracle_mod, monkeypatch, shape):
    # 20,000 variables: the first epoch's candidates overflow their slots under
    # 14,-2 and 13,-1 (fallback scan), the later ones take the sorted check
    monkeypatch.setenv("AMC_SCAN_TAIL", shape)
    ks, var = workloads.trace_zipf(3 * (1 << 20) + 5, 20_000, seed=97, device="cuda")
    check(amc, oracle_mod, ks.cpu().numpy(), var.cpu().numpy(), 20_000)


def test_long_run_across_sort_tiles(amc, oracle_mod, monkeypatch):
    # a tenth of the ops are CPU reads and writes of variable 7 (and no other
    # op is), so it never faults: in the last epoch its ~97,000 candidates span
    # many 4,096-pair tiles of the sorted check (the carry between tiles),
    # beside a Zipf background; the earlier epochs overflow into the fallback
    monkeypatch.setenv("AMC_SCAN_TAIL", "15,-2")
    rng = np.random.default_rng(98)
    nv = 40_000
    ks, var = workloads.trace_random(rng, 1_500_001, nv, zipf_s=1.05)
    var[var == 7] = 8
    hot = rng.random(ks.size) < 0.1
    ks[hot] = rng.integers(0, 2, int(hot.sum())).astype(np.uint8)     # CPU r / w
    var[hot] = 7
    check(amc, oracle_mod, ks, var, nv)


def test_first_part_with_faults_and_initial_statuses(amc, oracle_mod, monkeypatch):
    # first part 2^16 ops over 20,000 variables with every initial status,
    # uniform ids (about three ops per variable there), epochs of 2^16 ops
    monkeypatch.setenv("AMC_SCAN_TAIL", "16,16")
    rng = np.random.default_rng(99)
    nv = 20_000
    ks, var = workloads.trace_random(rng, 400_000, nv)
    init = rng.integers(0, 5, nv).astype(np.uint8)
    check(amc, oracle_mod, ks, var, nv, init)


def test_bad_input_in_the_first_part(amc, monkeypatch):
    monkeypatch.setenv("AMC_SCAN_TAIL", "14,14")
    dev = torch.device("cuda")
    n, nv = 50_000, 20_000
    ks = torch.zeros(n, dtype=torch.uint8, device=dev)
    var = torch.arange(n, dtype=torch.int32, device=dev) % nv
    var[100] = -3                                  # id out of range, in the first part
    amc.check_trace(ks, var, nv)
    assert amc.sync_status() == amc.E_RANGE
    var[100] = 5
    ks[2_000] = 0x68                               # malformed byte
    amc.check_trace(ks, var, nv)
    assert amc.sync_status() == amc.E_INVALID
    ks[2_000] = 0x16                               # GT (GPU side) in a plain check, not before its EN
    amc.check_trace(ks, var, nv)
    assert amc.sync_status() == amc.E_INVALID
    assert amc.sync_status() == 0


def test_many_long_lived_variables(amc, oracle_mod, monkeypatch):
    # first part 2^16 ops, epochs of 2^18: a Zipf background over 40,000
    # variables, plus 10,000 variables that only see CPU reads, writes and
    # Noops (never stuck), 200 of them per epoch with 1..1,000 ops each, so
    # runs of every length cross the sorted check's tiles at every offset;
    # variable 49,999 gets 1,024 ops in the second epoch and 1,025 in the third
    monkeypatch.setenv("AMC_SCAN_TAIL", "16,18")
    rng = np.random.default_rng(96)
    nv, n = 50_000, 1_200_000
    ks, var = workloads.trace_random(rng, n, 40_000, zipf_s=1.05)
    S, E = 1 << 16, 1 << 18
    for j, e0 in enumerate(range(S, n, E)):
        e1 = min(e0 + E, n)
        ids = rng.choice(np.arange(40_000, 49_999), size=200, replace=False)
        kk = rng.integers(1, 1001, size=200)
        extra = {1: 1024, 2: 1025}.get(j, 0)
        tot = int(kk.sum()) + extra
        if tot > (e1 - e0) // 2:
            kk = np.maximum(1, kk * ((e1 - e0) // 2) // max(tot, 1))
            tot = int(kk.sum()) + extra
        pos = e0 + rng.choice(e1 - e0, size=tot, replace=False)
        who = np.concatenate([np.repeat(ids, kk), np.full(extra, 49_999)]).astype(np.int32)
        rng.shuffle(who)
        var[pos] = who
        ks[pos] = rng.choice(np.array([0x00, 0x01, 0x04], np.uint8), size=tot)
    check(amc, oracle_mod, ks, var, nv)


def test_graph_replay_on_a_side_stream(amc, oracle_mod, monkeypatch):
    # once a size class is tuned, checks on a non-default stream replay a
    # captured graph of the launch sequence: repeated calls on the same buffers
    # with new contents each time (and a changed knob, which captures anew)
    # must still give the oracle's outputs
    dev = torch.device("cuda")
    n, nv = 300_011, 40_000
    s = torch.cuda.Stream()
    ks_d = torch.empty(n, dtype=torch.uint8, device=dev)
    var_d = torch.empty(n, dtype=torch.int32, device=dev)
    out = dict(step_status=torch.empty(n, dtype=torch.uint8, device=dev),
               final_status=torch.empty(nv, dtype=torch.uint8, device=dev),
               var_first_fault=torch.empty(nv, dtype=torch.int32, device=dev),
               first_fault=torch.empty(1, dtype=torch.int64, device=dev))
    ws = torch.empty(amc.trace_workspace_bytes(n, nv) + 256, dtype=torch.uint8, device=dev)
    ws = ws[(-ws.data_ptr()) % 256:]
    rng = np.random.default_rng(97)
    for shape in ("14,16", "14,16", "14,16", "15,-2", "15,-2"):
        monkeypatch.setenv("AMC_SCAN_TAIL", shape)
        ks, var = workloads.trace_random(rng, n, nv, zipf_s=1.05)
        s.wait_stream(torch.cuda.current_stream())
        with torch.cuda.stream(s):
            ks_d.copy_(torch.from_numpy(ks))
            var_d.copy_(torch.from_numpy(var))
            amc.check_trace(ks_d, var_d, nv, out=out, workspace=ws, stream=s)
        s.synchronize()
        assert amc.sync_status() == 0
        exp = oracle_mod.check_trace(ks, var, nv)
        assert np.array_equal(out["step_status"].cpu().numpy(), exp[0]), shape
        assert np.array_equal(out["final_status"].cpu().numpy(), exp[1]), shape
        assert np.array_equal(out["var_first_fault"].cpu().numpy(), exp[2]), shape
        assert int(out["first_fault"].cpu()[0]) == exp[3], shape


@pytest.mark.parametrize("n_vars", [16_385, 100_003])
def test_bucket_widths(amc, oracle_mod, monkeypatch, n_vars):
    # the epochs' candidates go to 128 buckets of the ids v with v mod 128 = b:
    # 129 ids per bucket (rows padded) at the smallest variable count the epoch
    # path takes, and a count that leaves the last buckets one id short
    monkeypatch.setenv("AMC_SCAN_TAIL", "14,-2")
    rng = np.random.default_rng(98)
    ks, var = workloads.trace_random(rng, 600_001, n_vars, zipf_s=1.05)
    check(amc, oracle_mod, ks, var, n_vars)
