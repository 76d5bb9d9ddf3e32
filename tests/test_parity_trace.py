"""GPU parity of amc_check_trace with the oracle, element by element.

Bit-exact on every step status, final status, per-variable first fault and
global first fault (integer work: no tolerance).  Sizes span several tiles of
4,096 ops and ragged tails; edge cases: empty trace, one op, one variable,
every op on one variable, var ids at the top of the range, initial statuses
including (I,I) and F, and faulty op bytes / ids reported by sync_status."""
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


def run_both(amc, oracle_mod, ks, var, n_vars, init=None):
    exp = oracle_mod.check_trace(ks, var, n_vars, init)
    dev = torch.device("cuda")
    out = amc.check_trace(torch.from_numpy(ks).to(dev), torch.from_numpy(var).to(dev), n_vars,
                          None if init is None else torch.from_numpy(init).to(dev))
    assert amc.sync_status() == 0
    got = (out["step_status"].cpu().numpy(), out["final_status"].cpu().numpy(),
           out["var_first_fault"].cpu().numpy(), int(out["first_fault"].cpu()[0]))
    return exp, got


def assert_same(exp, got):
    assert np.array_equal(exp[0], got[0]), np.nonzero(exp[0] != got[0])[0][:10]
    assert np.array_equal(exp[1], got[1]), np.nonzero(exp[1] != got[1])[0][:10]
    assert np.array_equal(exp[2], got[2]), np.nonzero(exp[2] != got[2])[0][:10]
    assert exp[3] == got[3]


def test_uniform_16_vars_seed0(amc, oracle_mod):
    ks, var, nv = workloads.trace_uniform(0)
    assert_same(*run_both(amc, oracle_mod, ks, var, nv))


@pytest.mark.parametrize("n_ops,n_vars,zipf", [
    (1, 1, None), (17, 1, None), (4095, 3, None), (4096, 16, None), (4097, 16, None),
    (3 * 4096 + 17, 5, None), (50_000, 1000, 1.05), (200_003, 1 << 20, 1.05),
    (300_000, 7, None), (131_072, 1 << 16, None), (100_000, 2, None)])
def test_random_traces(amc, oracle_mod, n_ops, n_vars, zipf):
    rng = np.random.default_rng(n_ops + n_vars)
    ks, var = workloads.trace_random(rng, n_ops, n_vars, kinds=(0, 1, 2, 3, 4, 5, 7), zipf_s=zipf)
    assert_same(*run_both(amc, oracle_mod, ks, var, n_vars))


@pytest.mark.parametrize("mix", ["benign", "faulty"])
def test_low_fault_traces(amc, oracle_mod, mix):
    # mostly writes / noops so that statuses stay non-stuck across many tiles
    rng = np.random.default_rng(3)
    p = [0.02, 0.6, 0.05, 0.05, 0.28] if mix == "benign" else [0.3, 0.3, 0.1, 0.1, 0.2]
    ks, var = workloads.trace_random(rng, 400_000, 300, p=p)
    assert_same(*run_both(amc, oracle_mod, ks, var, 300))


def test_one_variable_many_tiles(amc, oracle_mod):
    rng = np.random.default_rng(4)
    ks, var = workloads.trace_random(rng, 70_001, 1, p=[0.0, 0.5, 0.0, 0.0, 0.5])
    ks[-5:] = np.array([0, 16, 2, 3, 0], np.uint8)
    assert_same(*run_both(amc, oracle_mod, ks, var, 1))


def test_top_of_id_range(amc, oracle_mod):
    rng = np.random.default_rng(5)
    n_vars = (1 << 24) + 3
    ks, var = workloads.trace_random(rng, 20_000, 4)
    var = (n_vars - 1 - var).astype(np.int32)
    assert_same(*run_both(amc, oracle_mod, ks, var, n_vars))


def test_initial_statuses(amc, oracle_mod):
    rng = np.random.default_rng(6)
    ks, var = workloads.trace_random(rng, 60_000, 64)
    init = rng.integers(0, 5, 64).astype(np.uint8)
    assert_same(*run_both(amc, oracle_mod, ks, var, 64, init))


def test_empty_trace(amc, oracle_mod):
    ks = np.zeros(0, np.uint8)
    var = np.zeros(0, np.int32)
    assert_same(*run_both(amc, oracle_mod, ks, var, 9))


def test_repeatable(amc):
    ks, var = workloads.trace_zipf(300_000, 1 << 20, seed=9, device="cuda")
    a = amc.check_trace(ks, var, 1 << 20)
    s1 = a["step_status"].clone()
    b = amc.check_trace(ks, var, 1 << 20)
    assert torch.equal(s1, b["step_status"])
    assert amc.sync_status() == 0


def test_bad_inputs_reported(amc):
    dev = torch.device("cuda")
    ks = torch.tensor([0, 1, 2], dtype=torch.uint8, device=dev)
    var = torch.tensor([0, 5, 1], dtype=torch.int32, device=dev)
    amc.check_trace(ks, var, 4)
    assert amc.sync_status() == amc.E_RANGE
    ks = torch.tensor([0, 0x21, 2], dtype=torch.uint8, device=dev)
    var = torch.tensor([0, 1, 1], dtype=torch.int32, device=dev)
    amc.check_trace(ks, var, 4)
    assert amc.sync_status() == amc.E_INVALID
    ks = torch.tensor([6, 7], dtype=torch.uint8, device=dev)        # GT needs the guarded call
    var = torch.tensor([0, 1], dtype=torch.int32, device=dev)
    amc.check_trace(ks, var, 4)
    assert amc.sync_status() == amc.E_INVALID
    assert amc.sync_status() == 0


def test_guarded_trace_from_vectorpu(amc, oracle_mod):
    w = workloads.vectorpu_calls(seed=21, n_arrays=64, space=1 << 14, n_calls=20_000,
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


def test_zipf_trace_full_size(amc, oracle_mod):
    """The 2^30-op, 2^20-var Zipf workload in the launch configuration the
    benchmark times, every output checked against the oracle."""
    n_ops, n_vars = 1 << 30, 1 << 20
    ks, var = workloads.trace_zipf(n_ops, n_vars, seed=1, device="cuda")
    out = amc.check_trace(ks, var, n_vars)
    assert amc.sync_status() == 0
    ks_h, var_h = ks.cpu().numpy(), var.cpu().numpy()
    del ks, var
    step = out["step_status"].cpu().numpy()
    final = out["final_status"].cpu().numpy()
    vff = out["var_first_fault"].cpu().numpy()
    ff = int(out["first_fault"].cpu()[0])
    del out
    torch.cuda.empty_cache()
    e_step, e_final, e_vff, e_ff = oracle_mod.check_trace(ks_h, var_h, n_vars)
    assert np.array_equal(e_final, final)
    assert np.array_equal(e_vff, vff)
    assert e_ff == ff
    assert np.array_equal(e_step, step)


def test_autotune_cache_file(tmp_path):
    """The first call of a shape times the candidate launch shapes and records
    the choice; outputs are identical whichever candidate runs."""
    import subprocess
    import sys
    cache = tmp_path / "tune.txt"
    code = (
        "import sys; sys.path.insert(0, '.'); import torch, numpy as np, workloads, oracle;"
        "import paper_1910_11110_gb300 as amc; amc.build();"
        "ks, var = workloads.trace_zipf(300_000, 1 << 16, seed=4, device='cuda');"
        "a = amc.check_trace(ks, var, 1 << 16); b = amc.check_trace(ks, var, 1 << 16);"
        "assert amc.sync_status() == 0;"
        "e = oracle.check_trace(ks.cpu().numpy(), var.cpu().numpy(), 1 << 16);"
        "assert np.array_equal(a['step_status'].cpu().numpy(), e[0]);"
        "assert torch.equal(a['step_status'], b['step_status'])")
    env = dict(__import__("os").environ, AMC_AUTOTUNE_CACHE=str(cache))
    r = subprocess.run([sys.executable, "-c", code], cwd=__import__("os").path.dirname(__import__("os").path.dirname(__file__)),
                       env=env, capture_output=True, text=True, timeout=300)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = cache.read_text().split()
    assert lines and lines[0].startswith("trace:")


@pytest.mark.parametrize("fb", ["-1", "1048576", "-2"])
@pytest.mark.parametrize("group", ["1", "-2"])
def test_initial_statuses_every_bitmap_mode(amc, oracle_mod, monkeypatch, fb, group):
    # variables that are F from the start fault nowhere inside the trace, whether
    # or not the stuck bitmap (none / shared memory / through L1) filters them
    monkeypatch.setenv("AMC_SCAN_FB_BITS", fb)
    monkeypatch.setenv("AMC_SCAN_GROUP", group)
    rng = np.random.default_rng(36)
    ks, var = workloads.trace_random(rng, 90_000, 64)
    init = rng.integers(0, 5, 64).astype(np.uint8)
    assert (init == 4).any()
    assert_same(*run_both(amc, oracle_mod, ks, var, 64, init))


@pytest.mark.parametrize("group", ["1", "-2", "16"])
def test_shared_window_with_l1_bitmap(amc, oracle_mod, monkeypatch, group):
    # stuck bits of the first 4,096 variables in shared memory, the others
    # read through L1: both lookups in one warp, stale copies only conservative
    monkeypatch.setenv("AMC_SCAN_FB_BITS", "-4096")
    monkeypatch.setenv("AMC_SCAN_GROUP", group)
    rng = np.random.default_rng(37)
    ks, var = workloads.trace_random(rng, 700_001, 1 << 16, zipf_s=1.05)
    assert_same(*run_both(amc, oracle_mod, ks, var, 1 << 16))
    init = rng.integers(0, 5, 1 << 16).astype(np.uint8)
    assert_same(*run_both(amc, oracle_mod, ks, var, 1 << 16, init))


@pytest.mark.parametrize("n_ops,n_vars", [(0, 5), (1, 1), (31, 3), (32, 16), (33, 16), (4096, 16), (4097, 2048),
                                          (65536, 2048), (65536, 1), (50_000, 700)])
def test_small_traces_one_cta(amc, oracle_mod, n_ops, n_vars):
    # traces of at most 2^16 ops over at most 2,048 variables are checked by
    # one CTA; every kind incl. EN, initial statuses incl. (I,I) and F
    rng = np.random.default_rng(n_ops * 7 + n_vars)
    ks, var = workloads.trace_random(rng, n_ops, n_vars, kinds=(0, 1, 2, 3, 4, 5, 7))
    init = rng.integers(0, 5, n_vars).astype(np.uint8)
    for ini in (None, init):
        exp = oracle_mod.check_trace(ks, var, n_vars, ini)
        dev = torch.device("cuda")
        out = amc.check_trace(torch.from_numpy(ks).to(dev), torch.from_numpy(var).to(dev), n_vars,
                              None if ini is None else torch.from_numpy(ini).to(dev))
        assert amc.sync_status() == 0
        assert np.array_equal(out["step_status"].cpu().numpy(), exp[0])
        assert np.array_equal(out["final_status"].cpu().numpy(), exp[1])
        assert np.array_equal(out["var_first_fault"].cpu().numpy(), exp[2])
        assert int(out["first_fault"].cpu()[0]) == exp[3]


def test_small_trace_bad_input(amc):
    dev = torch.device("cuda")
    ks = torch.zeros(100, dtype=torch.uint8, device=dev)
    var = torch.zeros(100, dtype=torch.int32, device=dev)
    var[50] = 9
    amc.check_trace(ks, var, 8)
    assert amc.sync_status() == amc.E_RANGE
    var[50] = 1
    ks[7] = 6                                   # GT in a plain check
    amc.check_trace(ks, var, 8)
    assert amc.sync_status() == amc.E_INVALID
    ks[7] = 0x48                                # malformed byte
    amc.check_trace(ks, var, 8)
    assert amc.sync_status() == amc.E_INVALID
    assert amc.sync_status() == 0
