"""GPU parity of amc_check_batch_guarded (path-sensitive relation mode:
conditions isValid g / remIsValid g on a guard variable per program, opaque
conditions as both outcomes) with the oracle (oracle_check_batch_guarded):
every step mask, final mask and program first fault bit-exact.  Covers the
seeded guarded-program workload (full size and variants: deep nesting, every
condition on g, programs past the shared-memory variable count), hand-made
programs (the guarded transfer of Fig. sem-AM, unreachable branches and loop
bodies, a loop that is never left, a stuck guard), the reduction to the
opaque relation mode, and malformed inputs."""
import numpy as np
import pytest
import torch

import workloads

pytestmark = pytest.mark.gpu
IF, ELSE, WHILE, END = 8, 9, 10, 11
R, W, PUSH, PULL, NOOP = 0, 1, 2, 3, 4


@pytest.fixture(scope="module")
def amc():
    import paper_1910_11110_gb300 as m
    m.build()
    return m


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def run(amc, b):
    out = amc.check_batch_guarded(dev(b["tok"]), dev(b["payload"]), dev(b["prog_tok_off"]), dev(b["prog_nvars"]),
                                  dev(b["prog_guard"]))
    code = amc.sync_status()
    return {k: v.cpu().numpy() for k, v in out.items()}, code


def compare(amc, oracle_mod, b):
    step, final, pff = oracle_mod.check_batch_guarded(b["tok"], b["payload"], b["prog_tok_off"], b["prog_nvars"],
                                                      b["prog_guard"])
    got, code = run(amc, b)
    assert code == 0
    bad = np.nonzero(got["step_mask"] != step)[0]
    assert bad.size == 0, bad[:10]
    assert np.array_equal(got["final_mask"], final)
    assert np.array_equal(got["prog_first_fault"], pff)


def test_guarded_workload_full_size(amc, oracle_mod):
    """20,000 programs over 16-256 variables (seed 7)."""
    compare(amc, oracle_mod, workloads.programs_guarded())


@pytest.mark.parametrize("kw", [
    dict(n_progs=300, seed=71, median=300.0, vars_lo=1, vars_hi=4, p_if=0.3, p_while=0.2),
    dict(n_progs=200, seed=72, median=500.0, vars_lo=2, vars_hi=40, p_cond=(0.0, 0.5, 0.5), p_if=0.25),
    dict(n_progs=100, seed=73, median=100.0, vars_lo=3, vars_hi=8, p_if=0.3, p_while=0.3, max_depth=8, max_branch=6,
         max_body=6),
    dict(n_progs=30, seed=74, median=2000.0, vars_lo=1100, vars_hi=3000),
    dict(n_progs=50, seed=75, median=5000.0, vars_lo=64, vars_hi=512, p_cond=(1.0, 0.0, 0.0)),
])
def test_guarded_batches(amc, oracle_mod, kw):
    compare(amc, oracle_mod, workloads.programs_guarded(**kw))


def concat(progs):
    tok = np.concatenate([np.asarray(p[0], np.uint8) for p in progs])
    pay = np.concatenate([np.asarray(p[1], np.int32) for p in progs])
    off = np.concatenate([[0], np.cumsum([len(p[0]) for p in progs])]).astype(np.int64)
    return dict(tok=tok, payload=pay, prog_tok_off=off, prog_nvars=np.array([p[2] for p in progs], np.int32),
                prog_guard=np.array([p[3] for p in progs], np.int32))


def test_hand_made_programs(amc, oracle_mod):
    progs = [
        # guarded transfer of Fig. sem-AM after an opaque If (x = 0, guard x# = 1)
        ([IF, W, W, ELSE, W | 16, W | 16, END, IF | 16, NOOP, ELSE, PULL, PULL, END, R],
         [2, 0, 1, 2, 0, 1, 0, 1, 0, 2, 0, 1, 0, 0], 2, 1),
        # While (isValid g) { GPU w g }: once round, leaves (I,V)
        ([WHILE | 16, W | 16, END], [1, 0, 0], 1, 0),
        # While (remIsValid g) on a (V,I) g: body unreachable
        ([WHILE | 32, R | 16, END], [1, 1, 0], 2, 0),
        # a loop never left: nothing after it reachable
        ([W | 16, WHILE | 32, R | 16, END, R], [0, 1, 1, 0, 1], 2, 0),
        # a stuck guard ends its paths at the next condition
        ([IF, R | 16, ELSE, NOOP, END, IF | 16, W, ELSE, W, END], [1, 0, 1, 0, 0, 1, 1, 1, 1, 0], 2, 0),
        # empty program, empty branches, no guard
        ([], [], 1, -1),
        ([IF, ELSE, END, WHILE, END], [0, 0, 0, 0, 0], 1, -1),
    ]
    b = concat(progs)
    compare(amc, oracle_mod, b)
    got, _ = run(amc, b)
    assert got["prog_first_fault"][0] == -1           # the guarded transfer never gets stuck


def test_opaque_conditions_equal_relation_mode(amc, oracle_mod):
    b = workloads.programs(400, seed=76, median=400.0, vars_lo=2, vars_hi=50, p_if=0.2, p_while=0.1)
    b["prog_guard"] = np.full(400, -1, np.int32)
    compare(amc, oracle_mod, b)
    got, _ = run(amc, b)
    plain = amc.check_batch(dev(b["tok"]), dev(b["payload"]), dev(b["prog_tok_off"]), dev(b["prog_nvars"]))
    assert amc.sync_status() == 0
    assert np.array_equal(plain["step_mask"].cpu().numpy(), got["step_mask"])
    assert np.array_equal(plain["final_mask"].cpu().numpy(), got["final_mask"])


@pytest.mark.parametrize("case,code", [
    ("condition_without_guard", "E_INVALID"), ("guard_out_of_range", "E_INVALID"), ("condition_3", "E_INVALID"),
    ("var_out_of_range", "E_RANGE"), ("unbalanced", "E_INVALID"),
])
def test_malformed_reported(amc, case, code):
    tok, pay, nv, g = [IF | 16, NOOP, ELSE, NOOP, END], [1, 0, 1, 0, 0], 2, 0
    if case == "condition_without_guard":
        g = -1
    elif case == "guard_out_of_range":
        g = 2
    elif case == "condition_3":
        tok = [IF | 48, NOOP, ELSE, NOOP, END]
    elif case == "var_out_of_range":
        pay = [1, 5, 1, 0, 0]
    elif case == "unbalanced":
        tok, pay = [IF | 16, NOOP], [1, 0]
    assert amc.sync_status() == 0
    _, got = run(amc, concat([(tok, pay, nv, g)]))
    assert got == getattr(amc, code)
    assert amc.sync_status() == 0
