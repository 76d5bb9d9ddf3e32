"""The oracle's static well-declaredness check (Section 3.3, Definitions
"Occurs in all execution paths" and "Well-declared program"; Section 3.5,
"Well-declared program with array access"), pinned by the paper's examples,
by brute-force enumeration of the execution paths of small bodies, and by the
property the definitions exist for: a well-declared program, translated by
Fig. sem-AM and run, never gets stuck (Theorem Progress for well-declared
programs)."""
import itertools
import json
import os

import numpy as np
import pytest

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "section3_3_well_declared.json")
IF, ELSE, WHILE, END = 8, 9, 10, 11
R, W, RW = 1, 2, 3


def pack(arrays, calls):
    """arrays: locations per array; calls: [(am [(array, mode | side << 4)],
    body [(byte, payload)])] -> the CSR arguments of oracle.well_declared."""
    alo = np.zeros(len(arrays) + 1, np.int64)
    alo[1:] = np.cumsum(arrays)
    owner = np.repeat(np.arange(len(arrays)), arrays).astype(np.int32)
    cto, cao, tok, pay, aa, am = [0], [0], [], [], [], []
    for decl, body in calls:
        for b, p in body:
            tok.append(b)
            pay.append(p)
        for a, m in decl:
            aa.append(a)
            am.append(m)
        cto.append(len(tok))
        cao.append(len(aa))
    return (alo, owner, np.array(cto, np.int64), np.array(tok, np.uint8), np.array(pay, np.int32),
            np.array(cao, np.int64), np.array(aa, np.int32), np.array(am, np.uint8))


def test_paper_examples(oracle_mod):
    cases = json.load(open(GOLDEN))["cases"]
    for case in cases:
        calls = [(c["am"], c["body"]) for c in case["calls"]]
        viol, bad, unmet = oracle_mod.well_declared(*pack(case["arrays"], calls))
        for c, (v, b, u) in zip(case["calls"], zip(viol, bad, unmet)):
            assert [int(v), int(b), int(u)] == c["expect"], (case["cite"], c)


# ---- random bodies and brute-force path enumeration -------------------------
def random_body(rng, n_locs, depth=0, budget=None):
    """A random statement list over n_locs locations (reads, writes and Noops on
    either side; Ifs and Whiles nested at most 3 deep)."""
    if budget is None:
        budget = [int(rng.integers(1, 9))]
    items = []
    while budget[0] > 0:
        budget[0] -= 1
        x = rng.random()
        if depth < 3 and x < 0.2:
            items.append(("if", random_body(rng, n_locs, depth + 1, [int(rng.integers(0, 4))]),
                          random_body(rng, n_locs, depth + 1, [int(rng.integers(0, 4))])))
        elif depth < 3 and x < 0.3:
            items.append(("while", random_body(rng, n_locs, depth + 1, [int(rng.integers(0, 4))])))
        else:
            kind = int(rng.choice([0, 1, 4], p=[0.3, 0.6, 0.1]))
            items.append(("op", kind | int(rng.integers(0, 2)) << 4, int(rng.integers(0, n_locs))))
    return items


def tokens(items):
    out = []
    for it in items:
        if it[0] == "op":
            out.append((it[1], it[2]))
        elif it[0] == "if":
            a, b = tokens(it[1]), tokens(it[2])
            out += [(IF, len(a))] + a + [(ELSE, len(b))] + b + [(END, 0)]
        else:
            a = tokens(it[1])
            out += [(WHILE, len(a))] + a + [(END, 0)]
    return out


def paths(items, unroll=2):
    """Every execution path (list of op tuples), a While run 0..unroll times."""
    res = [[]]
    for it in items:
        if it[0] == "op":
            alts = [[(it[1], it[2])]]
        elif it[0] == "if":
            alts = paths(it[1], unroll) + paths(it[2], unroll)
        else:
            body = paths(it[1], unroll)
            alts = [[]]
            for k in range(1, unroll + 1):
                for combo in itertools.product(body, repeat=k):
                    alts.append([op for p in combo for op in p])
        res = [p + a for p in res for a in alts]
    return res


@pytest.mark.parametrize("seed", range(6))
def test_obligations_by_path_enumeration(oracle_mod, seed):
    # for every W declaration: each location of the array is written on that
    # side on every enumerated path <=> no unmet obligation for that array
    rng = np.random.default_rng(400 + seed)
    arrays = [1, 2, 1]
    owner = np.repeat(np.arange(3), arrays)
    calls, exp_unmet = [], []
    for _ in range(60):
        body = random_body(rng, 4)
        decl = [(a, int(rng.choice([R, W, RW])) | int(rng.integers(0, 2)) << 4)
                for a in rng.choice(3, size=int(rng.integers(1, 4)), replace=False)]
        ps = paths(body)
        unmet = -1
        for a, m in decl:
            if m & 15 != W:
                continue
            side = m >> 4
            for loc in np.nonzero(owner == a)[0]:
                if not all(any(b == (1 | side << 4) and p == loc for b, p in path) for path in ps):
                    unmet = a if unmet < 0 else min(unmet, a)
                    break
        calls.append((decl, tokens(body)))
        exp_unmet.append(unmet)
    viol, bad, unmet = oracle_mod.well_declared(*pack(arrays, calls))
    assert list(unmet) == exp_unmet
    assert [bool(v & 8) for v in viol] == [u >= 0 for u in exp_unmet]
    assert sum(u >= 0 for u in exp_unmet) > 5 and sum(u < 0 for u in exp_unmet) > 5


def test_accepted_straight_line_programs_never_fault(oracle_mod):
    # Theorem Progress for well-declared programs: scalar variables (arrays of
    # one location), straight-line bodies; every call the check accepts is
    # translated by Fig. sem-AM (R: GT x, EN x#; W: w x#; RW: both) and run in
    # trace mode from (V,I): no op gets stuck.  Calls it rejects are skipped.
    rng = np.random.default_rng(41)
    n = 6
    accepted = 0
    ks, var = [], []
    for _ in range(3000):
        side = int(rng.integers(0, 2))
        decl = [(int(a), int(rng.choice([R, W, RW])) | side << 4)
                for a in rng.choice(n, size=int(rng.integers(1, 4)), replace=False)]
        names = [a for a, _ in decl] + [int(rng.integers(0, n))]          # mostly declared variables
        body = [(int(rng.choice([0, 1])) | side << 4, int(rng.choice(names))) for _ in range(int(rng.integers(1, 5)))]
        viol, _, _ = oracle_mod.well_declared(*pack([1] * n, [(decl, body)]))
        if viol[0]:
            continue
        accepted += 1
        for a, m in decl:
            if m & 15 in (R, RW):
                ks += [6 | side << 4, 7 | side << 4]
                var += [a, n + a]
            if m & 15 in (W, RW):
                ks.append(1 | side << 4)
                var.append(n + a)
        for b, p in body:
            ks.append(b)
            var.append(p)
    assert accepted > 300
    step, final, vff, ff = oracle_mod.check_trace(np.array(ks, np.uint8), np.array(var, np.int32), 2 * n)
    assert ff == -1 and not (step == 4).any()


def test_rejects_malformed(oracle_mod):
    with pytest.raises(oracle_mod.OracleError):        # unbalanced If
        oracle_mod.well_declared(*pack([1], [([(0, RW)], [(IF, 1), (1, 0)])]))
    with pytest.raises(oracle_mod.OracleError):        # GT is not a statement of a body
        oracle_mod.well_declared(*pack([1], [([(0, RW)], [(6, 0)])]))
    with pytest.raises(oracle_mod.OracleError):        # location out of range
        oracle_mod.well_declared(*pack([1], [([(0, RW)], [(1, 5)])]))
