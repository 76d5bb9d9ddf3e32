"""Pins of the oracle's trace mode against what the paper fixes (CPU only).

None of these checks re-types the oracle's unification code: they use the
paper's worked examples, its prose statements about each effect, Property
Safety, the stated equivalence Pull = rem Push, and structural facts of the
sequential semantics (per-variable independence, splitting a trace).
"""
import json
import os

import numpy as np
import pytest

import workloads

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")
R_, W_, PUSH, PULL, NOOP, PW = 0, 1, 2, 3, 4, 5
F = 4
VI, IV, VV, II = 1, 2, 3, 0


def cpu(s):
    return s & 1


def gpu(s):
    return (s >> 1) & 1


def test_unification_example(oracle_mod):
    g = json.load(open(os.path.join(GOLDEN, "section3_examples.json")))["unification_example"]
    for c in g["cases"]:
        assert oracle_mod.apply(c["kind"], c["side"], c["pre"]) == c["post"], c


@pytest.mark.parametrize("name", ["stuck_example", "push_example"])
def test_section3_2_examples(oracle_mod, name):
    g = json.load(open(os.path.join(GOLDEN, "section3_examples.json")))[name]
    ks = np.array([k | s << 4 for k, s in g["ops"]], np.uint8)
    var = np.zeros(len(ks), np.int32)
    step, final, vff, ff = oracle_mod.check_trace(ks, var, 1)
    assert step.tolist() == g["status"]
    assert ff == g["first_fault"]
    assert final[0] == g["status"][-1]


def test_effect_prose(oracle_mod):
    """Section 3.1 prose about each effect, checked on every non-stuck status."""
    for s in range(4):
        # r requires local validity and leaves the status unchanged
        assert oracle_mod.apply(R_, 0, s) == (s if cpu(s) else F)
        # w needs no validity, makes the local copy valid and the remote invalid
        assert oracle_mod.apply(W_, 0, s) == VI
        # Push requires local validity and makes the distant copy valid
        assert oracle_mod.apply(PUSH, 0, s) == (VV if cpu(s) else F)
        # Pull is the symmetric operation
        assert oracle_mod.apply(PULL, 0, s) == (VV if gpu(s) else F)
        # Noop does nothing
        assert oracle_mod.apply(NOOP, 0, s) == s
        assert oracle_mod.apply(NOOP, 1, s) == s
    for k in range(6):
        for side in (0, 1):
            assert oracle_mod.apply(k, side, F) == F      # stuck stays stuck


def _swap(s):
    return s if s == F else ((s & 1) << 1) | (s >> 1)


def test_remote_is_symmetric(oracle_mod):
    """Remote Effect swaps the pair (Fig. Opsem); Pull is rem Push (Section 3.2)."""
    for s in range(5):
        for k in range(6):
            assert oracle_mod.apply(k, 1, s) == _swap(oracle_mod.apply(k, 0, _swap(s)))
        assert oracle_mod.apply(PULL, 0, s) == oracle_mod.apply(PUSH, 1, s)
        assert oracle_mod.apply(PUSH, 0, s) == oracle_mod.apply(PULL, 1, s)


def test_progress_stuck_iff_requirement_fails(oracle_mod):
    """Property Progress: a step is stuck exactly when the accessed side the
    effect requires is invalid.  r and Push need the side they run on, Pull
    needs the other side, w and Noop need nothing."""
    need = {R_: "own", PUSH: "own", PULL: "other", W_: None, NOOP: None, PW: None}
    for s in range(4):
        for k, req in need.items():
            for side in (0, 1):
                own = cpu(s) if side == 0 else gpu(s)
                other = gpu(s) if side == 0 else cpu(s)
                ok = True if req is None else bool(own if req == "own" else other)
                assert (oracle_mod.apply(k, side, s) != F) == ok, (k, side, s)


def test_safety_no_ii_from_initial_state(oracle_mod):
    """Property Safety: core ops from sigma_0 never reach (I,I)."""
    rng = np.random.default_rng(11)
    for _ in range(20):
        ks, var = workloads.trace_random(rng, 2000, 7)
        step, final, _, _ = oracle_mod.check_trace(ks, var, 7)
        assert not np.any(step == II)
        assert not np.any(final == II)


def test_partial_write_can_reach_ii(oracle_mod):
    # pw is not a core op; Safety does not cover it: (I,V) partly written on the CPU
    assert oracle_mod.apply(PW, 0, IV) == II


def test_per_variable_independence(oracle_mod):
    """Effect / Remote Effect touch only sigma(x): each variable's subsequence
    checked alone gives the same statuses."""
    rng = np.random.default_rng(5)
    ks, var = workloads.trace_random(rng, 3000, 9, zipf_s=1.05)
    step, final, vff, ff = oracle_mod.check_trace(ks, var, 9)
    for v in range(9):
        idx = np.nonzero(var == v)[0]
        s2, f2, vff2, _ = oracle_mod.check_trace(ks[idx], np.zeros(len(idx), np.int32), 1)
        assert np.array_equal(s2, step[idx])
        assert f2[0] == final[v]
        assert (vff2[0] == -1 and vff[v] == -1) or idx[vff2[0]] == vff[v]
    faults = vff[vff >= 0]
    assert ff == (faults.min() if len(faults) else -1)


def test_split_trace_equals_whole(oracle_mod):
    """Sequencing is associative (Section 3.2): the final store of a prefix is
    the initial store of the rest."""
    rng = np.random.default_rng(6)
    ks, var = workloads.trace_random(rng, 5000, 13, p=[.4, .2, .15, .15, .1])
    step, final, vff, ff = oracle_mod.check_trace(ks, var, 13)
    for cut in (0, 1, 777, 4999, 5000):
        s1, f1, _, _ = oracle_mod.check_trace(ks[:cut], var[:cut], 13)
        s2, f2, _, _ = oracle_mod.check_trace(ks[cut:], var[cut:], 13, init_status=f1)
        assert np.array_equal(np.concatenate([s1, s2]), step)
        assert np.array_equal(f2, final)


def test_first_fault_definition(oracle_mod):
    rng = np.random.default_rng(8)
    ks, var = workloads.trace_random(rng, 4000, 16)
    step, final, vff, ff = oracle_mod.check_trace(ks, var, 16)
    for v in range(16):
        idx = np.nonzero(var == v)[0]
        fs = idx[step[idx] == F]
        assert vff[v] == (fs[0] if len(fs) else -1)
        if len(fs):                 # stuck is absorbing
            assert np.all(step[idx[idx >= fs[0]]] == F)


def test_initial_status_argument(oracle_mod):
    ks = np.array([R_ | 1 << 4, W_, R_ | 1 << 4], np.uint8)
    var = np.zeros(3, np.int32)
    step, *_ = oracle_mod.check_trace(ks, var, 1, init_status=np.array([VV], np.uint8))
    assert step.tolist() == [VV, VI, F]
    step, *_ = oracle_mod.check_trace(ks, var, 1, init_status=np.array([F], np.uint8))
    assert step.tolist() == [F, F, F]


def test_rejects_malformed(oracle_mod):
    with pytest.raises(oracle_mod.OracleError):
        oracle_mod.check_trace(np.array([0], np.uint8), np.array([3], np.int32), 2)
    with pytest.raises(oracle_mod.OracleError):
        oracle_mod.check_trace(np.array([0x20], np.uint8), np.array([0], np.int32), 2)
    with pytest.raises(oracle_mod.OracleError):   # GT without its EN
        oracle_mod.check_trace(np.array([6], np.uint8), np.array([0], np.int32), 2)


def test_empty_trace(oracle_mod):
    step, final, vff, ff = oracle_mod.check_trace(np.zeros(0, np.uint8), np.zeros(0, np.int32), 4)
    assert len(step) == 0 and final.tolist() == [VI] * 4 and ff == -1 and vff.tolist() == [-1] * 4


def test_uniform_workload_statistics(oracle_mod):
    """The uniform 16-var workload: most per-step outputs are stuck."""
    ks, var, nv = workloads.trace_uniform(0)
    step, final, vff, ff = oracle_mod.check_trace(ks, var, nv)
    assert 0.9 < np.mean(step == F) < 1.0
    assert ff >= 0


@pytest.mark.parametrize("threads", [1, 3, 7])
def test_sharded_driver_equals_whole(oracle_mod, threads):
    # the multi-thread CPU baseline: each thread takes the variables v % T == t
    # (statuses depend only on a variable's own ops); its outputs must be
    # those of the one-thread check on every position and variable
    rng = np.random.default_rng(31 + threads)
    ks, var = workloads.trace_random(rng, 50_001, 997, zipf_s=1.05)
    exp = oracle_mod.check_trace(ks, var, 997)
    got = oracle_mod.check_trace_sharded(ks, var, 997, threads)
    for e, g in zip(exp[:3], got[:3]):
        assert np.array_equal(e, g)
    assert exp[3] == got[3]
