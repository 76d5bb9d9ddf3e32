"""Pins of the oracle's relation mode (If = union of branches, While = closure).

The reference here is brute force: every execution path of a tiny program
(both branches of each If, each While unrolled 0..5 times, which is enough
for a closure over five statuses) is run through the straight-line trace mode,
and the per-op status sets are the unions over all paths.  Conditions are
opaque (Section 3.2: the generic operator is assumed to succeed), so every
branch and every iteration count is a possible path (rules IF-True/IF-False,
While-True/While-False of Fig. Opsem).
"""
import itertools

import numpy as np
import pytest

F = 4
IF, ELSE, WHILE, END = 8, 9, 10, 11
UNROLL = 5
MAX_PATHS = 4000


def gen_node_list(rng, n_ops, n_vars, depth, max_depth):
    nodes = []
    while n_ops > 0:
        u = rng.random()
        if depth < max_depth and u < 0.2:
            t = int(rng.integers(0, min(3, n_ops) + 1))
            e = int(rng.integers(0, min(3, n_ops - t) + 1))
            nodes.append(("if", gen_node_list(rng, t, n_vars, depth + 1, max_depth),
                          gen_node_list(rng, e, n_vars, depth + 1, max_depth)))
            n_ops -= t + e
        elif depth < max_depth and u < 0.35:
            b = int(rng.integers(1, min(3, n_ops) + 1))
            nodes.append(("while", gen_node_list(rng, b, n_vars, depth + 1, max_depth)))
            n_ops -= b
        else:
            k = int(rng.integers(0, 5))
            s = int(rng.integers(0, 2))
            nodes.append(("op", k | s << 4, int(rng.integers(0, n_vars))))
            n_ops -= 1
    return nodes


def serialize(nodes, tok, pay):
    """Token stream; records for each op node its token index."""
    for nd in nodes:
        if nd[0] == "op":
            tok.append(nd[1]); pay.append(nd[2])
        elif nd[0] == "if":
            i = len(tok); tok.append(IF); pay.append(0)
            serialize(nd[1], tok, pay)
            e = len(tok); tok.append(ELSE); pay.append(0)
            serialize(nd[2], tok, pay)
            pay[i] = e - i - 1
            pay[e] = len(tok) - e - 1
            tok.append(END); pay.append(0)
        else:
            i = len(tok); tok.append(WHILE); pay.append(0)
            serialize(nd[1], tok, pay)
            pay[i] = len(tok) - i - 1
            tok.append(END); pay.append(0)


def index_nodes(nodes, start=0):
    """Attach token indices to op nodes (same walk as serialize)."""
    out = []
    i = start
    for nd in nodes:
        if nd[0] == "op":
            out.append(("op", nd[1], nd[2], i)); i += 1
        elif nd[0] == "if":
            i += 1
            t, i = index_nodes(nd[1], i)
            i += 1
            e, i = index_nodes(nd[2], i)
            i += 1
            out.append(("if", t, e))
        else:
            i += 1
            b, i = index_nodes(nd[1], i)
            i += 1
            out.append(("while", b))
    return out, i


def paths(nodes):
    """All execution paths as lists of (token index, op byte, var)."""
    acc = [[]]
    for nd in nodes:
        if nd[0] == "op":
            opts = [[(nd[3], nd[1], nd[2])]]
        elif nd[0] == "if":
            opts = paths(nd[1]) + paths(nd[2])
        else:
            body = paths(nd[1])
            opts = [[]]
            cur = [[]]
            for _ in range(UNROLL):
                cur = [a + b for a in cur for b in body]
                opts += cur
                if len(opts) > MAX_PATHS:
                    raise OverflowError
        acc = [a + b for a in acc for b in opts]
        if len(acc) > MAX_PATHS:
            raise OverflowError
    return acc


def brute_force(oracle_mod, nodes, n_tok, n_vars):
    inodes, _ = index_nodes(nodes)
    step = np.zeros(n_tok, np.uint8)
    final = np.zeros(n_vars, np.uint8)
    ff = -1
    for p in paths(inodes):
        idx = np.array([q[0] for q in p], np.int64)
        ks = np.array([q[1] for q in p], np.uint8)
        var = np.array([q[2] for q in p], np.int32)
        s, fin, vff, _ = oracle_mod.check_trace(ks, var, n_vars)
        for j in range(len(p)):
            step[idx[j]] |= 1 << int(s[j])
        final |= (1 << fin.astype(np.uint8)).astype(np.uint8)
        for v in range(n_vars):
            if vff[v] >= 0:
                t = int(idx[vff[v]])
                ff = t if ff < 0 else min(ff, t)
    return step, final, ff


@pytest.mark.parametrize("seed", range(24))
def test_relation_equals_path_enumeration(oracle_mod, seed):
    rng = np.random.default_rng(1000 + seed)
    n_vars = int(rng.integers(1, 4))
    for _ in range(10):
        nodes = gen_node_list(rng, int(rng.integers(1, 9)), n_vars, 0, 3)
        tok, pay = [], []
        serialize(nodes, tok, pay)
        try:
            bstep, bfinal, bff = brute_force(oracle_mod, nodes, len(tok), n_vars)
        except OverflowError:
            continue
        step, final, ff = oracle_mod.check_program(np.array(tok, np.uint8), np.array(pay, np.int32), n_vars)
        assert step.tolist() == bstep.tolist(), (tok, pay)
        assert final.tolist() == bfinal.tolist()
        assert ff == bff


def test_straight_line_reduces_to_trace_mode(oracle_mod):
    import workloads
    rng = np.random.default_rng(3)
    ks, var = workloads.trace_random(rng, 3000, 11)
    s, fin, vff, ff = oracle_mod.check_trace(ks, var, 11)
    m, mfin, mff = oracle_mod.check_program(ks, var, 11)
    assert np.array_equal(m, (1 << s.astype(np.int64)).astype(np.uint8))
    assert np.array_equal(mfin, (1 << fin.astype(np.int64)).astype(np.uint8))
    assert mff == ff


def test_empty_branches_and_loops(oracle_mod):
    # IF ELSE END with empty branches, WHILE with an empty body: identity
    tok = np.array([IF, ELSE, END, WHILE, END, 1 | 16], np.uint8)
    pay = np.array([0, 0, 0, 0, 0, 0], np.int32)
    step, final, ff = oracle_mod.check_program(tok, pay, 1)
    assert step.tolist() == [0, 0, 0, 0, 0, 1 << 2]
    assert final.tolist() == [1 << 2] and ff == -1


def test_while_closure_example(oracle_mod):
    # x starts (V,I); While { rem(w x); Push x } -- iteration 1: rem(w x) gives
    # (I,V), then local Push needs local validity and gets stuck.  The loop head
    # therefore sees {(V,I), stuck}; the body's sets are those from that set.
    tok = np.array([WHILE, 1 | 16, 2, END], np.uint8)
    pay = np.array([2, 0, 0, 0], np.int32)
    step, final, ff = oracle_mod.check_program(tok, pay, 1)
    assert step.tolist() == [0, (1 << 2) | (1 << F), 1 << F, 0]
    assert final.tolist() == [(1 << 1) | (1 << F)]
    assert ff == 2


def test_batch_matches_single_programs(oracle_mod):
    import workloads
    b = workloads.programs(30, seed=9, median=60.0, max_len=400, vars_lo=2, vars_hi=12)
    step, final, pff = oracle_mod.check_batch(b["tok"], b["payload"], b["prog_tok_off"], b["prog_nvars"])
    vo = np.concatenate([[0], np.cumsum(b["prog_nvars"])])
    for p in range(30):
        t0, t1 = b["prog_tok_off"][p], b["prog_tok_off"][p + 1]
        s, f, ff = oracle_mod.check_program(b["tok"][t0:t1], b["payload"][t0:t1], int(b["prog_nvars"][p]))
        assert np.array_equal(s, step[t0:t1])
        assert np.array_equal(f, final[vo[p]:vo[p + 1]])
        assert ff == pff[p]


def test_rejects_unbalanced(oracle_mod):
    with pytest.raises(oracle_mod.OracleError):
        oracle_mod.check_program(np.array([IF, 0], np.uint8), np.array([1, 0], np.int32), 1)
    with pytest.raises(oracle_mod.OracleError):
        oracle_mod.check_program(np.array([END], np.uint8), np.array([0], np.int32), 1)
