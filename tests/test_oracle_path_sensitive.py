"""Pins of the oracle's path-sensitive relation mode
(oracle_check_program_guarded): conditions isValid g / remIsValid g of
Fig. Opsem (rules valid, invalid, rem-valid, rem-invalid, IF-True/False,
While-True/False) evaluated on one guard variable g per program.

References: brute-force enumeration of the reachable concrete stores of tiny
programs (every store a tuple of statuses, If / While following the rules on
each store, loops iterated to their fixpoint over the finite store space),
whose per-token status sets the pair-set mode must reproduce exactly; the
opaque relation mode (oracle_check_program) when every condition is opaque;
the guarded transfer of Fig. sem-AM, which the path-sensitive mode proves
safe where the union of branches reports a spurious fault; and the
precision order (path-sensitive sets inside the opaque ones).
"""
import numpy as np
import pytest

IF, ELSE, WHILE, END = 8, 9, 10, 11
R, W, PUSH, PULL, NOOP = 0, 1, 2, 3, 4
II, VI, IV, VV, F = 0, 1, 2, 3, 4


def cond_holds(cond, s):
    """Rules valid / invalid (cond 1, local flag) and rem-valid / rem-invalid
    (cond 2, remote flag); None when no rule applies (a stuck status)."""
    if s == F:
        return None
    bit = 1 if cond == 1 else 2
    return bool(s & bit)


def brute(oracle_mod, tok, pay, nv, g, init=None):
    """Reachable concrete stores.  Returns (step_mask, final_mask, first_fault)."""
    n = len(tok)
    posts = [0] * n
    ff = [None]

    def run(lo, hi, S):
        i = lo
        while i < hi:
            t = int(tok[i])
            k, hb = t & 15, t >> 4
            if k <= 5:
                v = int(pay[i])
                out = set()
                for st in S:
                    post = oracle_mod.apply(k, hb, st[v])
                    if st[v] != F and post == F and (ff[0] is None or i < ff[0]):
                        ff[0] = i
                    posts[i] |= 1 << post
                    out.add(st[:v] + (post,) + st[v + 1:])
                S = out
                i += 1
            elif k == IF:
                e = i + 1 + int(pay[i])
                end = e + 1 + int(pay[e])
                if hb == 0:
                    St, Se = S, S
                else:
                    St = {st for st in S if cond_holds(hb, st[g]) is True}
                    Se = {st for st in S if cond_holds(hb, st[g]) is False}
                S = run(i + 1, e, St) | run(e + 1, end, Se)
                i = end + 1
            elif k == WHILE:
                end = i + 1 + int(pay[i])
                head = set(S)
                while True:
                    if hb == 0:
                        into = head
                    else:
                        into = {st for st in head if cond_holds(hb, st[g]) is True}
                    new = head | run(i + 1, end, into)
                    if new == head:
                        break
                    head = new
                S = head if hb == 0 else {st for st in head if cond_holds(hb, st[g]) is False}
                i = end + 1
            else:
                raise AssertionError("bad token")
        return S

    start = tuple(VI for _ in range(nv)) if init is None else tuple(init)
    S = run(0, n, {start})
    final = [0] * nv
    for st in S:
        for v in range(nv):
            final[v] |= 1 << st[v]
    # a variable whose every path ended keeps no status: the pair-set mode has
    # the same empty set
    return np.array(posts, np.uint8), np.array(final, np.uint8), -1 if ff[0] is None else ff[0]


def random_program(rng, nv, depth, budget, conds=(0, 1, 2)):
    toks = []

    def seq(d, n):
        for _ in range(n):
            u = rng.random()
            if d < depth and u < 0.2:
                c = int(rng.choice(conds))
                body = toks
                start = len(body)
                body.append([IF | (c << 4), 0])
                a = len(body)
                seq(d + 1, int(rng.integers(0, 4)))
                body[start][1] = len(body) - a
                e = len(body)
                body.append([ELSE, 0])
                b = len(body)
                seq(d + 1, int(rng.integers(0, 4)))
                body[e][1] = len(body) - b
                body.append([END, 0])
            elif d < depth and u < 0.35:
                c = int(rng.choice(conds))
                start = len(toks)
                toks.append([WHILE | (c << 4), 0])
                a = len(toks)
                seq(d + 1, int(rng.integers(0, 4)))
                toks[start][1] = len(toks) - a
                toks.append([END, 0])
            else:
                k = int(rng.choice([R, W, PUSH, PULL, NOOP], p=[0.25, 0.3, 0.15, 0.15, 0.15]))
                toks.append([k | (int(rng.integers(0, 2)) << 4), int(rng.integers(0, nv))])

    seq(0, budget)
    if not toks:
        toks = [[NOOP, 0]]
    t = np.array([x[0] for x in toks], np.uint8)
    p = np.array([x[1] for x in toks], np.int32)
    return t, p


@pytest.mark.parametrize("seed", range(40))
def test_matches_brute_force(oracle_mod, seed):
    rng = np.random.default_rng(1000 + seed)
    nv = int(rng.integers(1, 4))
    g = int(rng.integers(0, nv))
    tok, pay = random_program(rng, nv, depth=3, budget=int(rng.integers(3, 10)))
    step, final, ff = oracle_mod.check_program_guarded(tok, pay, nv, g)
    bstep, bfinal, bff = brute(oracle_mod, tok, pay, nv, g)
    ops = (tok & 15) <= 5
    assert np.array_equal(step[ops], bstep[ops]), (tok, pay, g)
    assert np.array_equal(final, bfinal)
    assert ff == bff


@pytest.mark.parametrize("seed", range(10))
def test_matches_brute_force_from_initial_sets(oracle_mod, seed):
    # initial statuses given per variable; the pair sets start as the product
    rng = np.random.default_rng(2000 + seed)
    nv = int(rng.integers(2, 4))
    g = int(rng.integers(0, nv))
    init = rng.integers(0, 5, nv)
    tok, pay = random_program(rng, nv, depth=2, budget=8)
    step, final, ff = oracle_mod.check_program_guarded(tok, pay, nv, g, init_mask=(1 << init).astype(np.uint8))
    bstep, bfinal, bff = brute(oracle_mod, tok, pay, nv, g, init=[int(x) for x in init])
    ops = (tok & 15) <= 5
    assert np.array_equal(step[ops], bstep[ops])
    assert np.array_equal(final, bfinal) and ff == bff


@pytest.mark.parametrize("seed", range(8))
def test_opaque_conditions_reduce_to_relation_mode(oracle_mod, seed):
    import workloads
    b = workloads.programs(20, seed=300 + seed, median=200.0, vars_lo=1, vars_hi=12, p_if=0.15, p_while=0.1)
    for p in range(20):
        a, z = b["prog_tok_off"][p], b["prog_tok_off"][p + 1]
        tok, pay, nv = b["tok"][a:z], b["payload"][a:z], int(b["prog_nvars"][p])
        exp = oracle_mod.check_program(tok, pay, nv)
        for g in (-1, nv - 1):
            got = oracle_mod.check_program_guarded(tok, pay, nv, g)
            assert np.array_equal(got[0], exp[0]) and np.array_equal(got[1], exp[1]) and got[2] == exp[2]


def test_guarded_transfer_of_fig_sem_am(oracle_mod):
    # x = 0, x# = 1 (the guard).  An opaque If leaves (x, x#) both (V,I) or
    # both (I,V); then [[R x#]] = if (isValid x#) Noop else (Pull x; Pull x#),
    # and the body's r x.  Path-sensitive: the Pull runs only on the (I,V)
    # paths, so nothing gets stuck and x ends (V,I) or (V,V); the union of
    # both branches (opaque condition) pulls from (V,I) too and reports it.
    tok = np.array([IF, W, W, ELSE, W | 16, W | 16, END,
                    IF | (1 << 4), NOOP, ELSE, PULL, PULL, END, R], np.uint8)
    pay = np.array([2, 0, 1, 2, 0, 1, 0,
                    1, 0, 2, 0, 1, 0, 0], np.int32)
    step, final, ff = oracle_mod.check_program_guarded(tok, pay, 2, 1)
    assert ff == -1
    assert step[10] == 1 << VV and step[11] == 1 << VV           # only (I,V) reaches the Pulls
    assert step[13] == (1 << VI) | (1 << VV)
    assert final[0] == (1 << VI) | (1 << VV) and final[1] == (1 << VI) | (1 << VV)
    opaque = tok.copy()
    opaque[7] = IF
    ostep, ofinal, off = oracle_mod.check_program_guarded(opaque, pay, 2, 1)
    assert off == 10 and ostep[13] & (1 << F)


def test_loop_exit_and_unreachable_code(oracle_mod):
    # while (isValid g) { GPU w g }: runs once from (V,I); leaves with (I,V)
    tok = np.array([WHILE | (1 << 4), W | 16, END], np.uint8)
    step, final, ff = oracle_mod.check_program_guarded(tok, np.array([1, 0, 0], np.int32), 1, 0)
    assert step[1] == 1 << IV and final[0] == 1 << IV and ff == -1
    # while (remIsValid g) on a (V,I) g: the body is never reached (empty sets)
    tok = np.array([WHILE | (2 << 4), R | 16, END], np.uint8)
    step, final, ff = oracle_mod.check_program_guarded(tok, np.array([1, 1, 0], np.int32), 2, 0)
    assert step[1] == 0 and ff == -1 and final[0] == 1 << VI and final[1] == 1 << VI
    # a loop that cannot be left (g stays (I,V)): its body faults (GPU r of a
    # (V,I) x), and nothing after it is reachable
    tok = np.array([W | 16, WHILE | (2 << 4), R | 16, END, R], np.uint8)
    step, final, ff = oracle_mod.check_program_guarded(tok, np.array([0, 1, 1, 0, 1], np.int32), 2, 0)
    assert ff == 2 and step[2] == 1 << F and step[4] == 0
    assert final[0] == 0 and final[1] == 0


def test_stuck_guard_ends_its_paths(oracle_mod):
    # g stuck on one branch (r on the GPU from (V,I)): no condition rule
    # applies to it, so the next If on g continues only the other paths
    tok = np.array([IF, R | 16, ELSE, NOOP, END, IF | (1 << 4), W, ELSE, W, END], np.uint8)
    pay = np.array([1, 0, 1, 0, 0, 1, 1, 1, 1, 0], np.int32)
    step, final, ff = oracle_mod.check_program_guarded(tok, pay, 2, 0)
    assert ff == 1
    assert final[0] == 1 << VI                 # the stuck paths of g ended at the condition
    assert step[6] == 1 << VI and step[8] == 0


@pytest.mark.parametrize("seed", range(6))
def test_more_precise_than_union(oracle_mod, seed):
    import workloads
    rng = np.random.default_rng(400 + seed)
    b = workloads.programs(30, seed=500 + seed, median=150.0, vars_lo=2, vars_hi=6, p_if=0.2, p_while=0.1)
    for p in range(30):
        a, z = b["prog_tok_off"][p], b["prog_tok_off"][p + 1]
        tok, pay, nv = b["tok"][a:z].copy(), b["payload"][a:z], int(b["prog_nvars"][p])
        st = (tok & 15 == IF) | (tok & 15 == WHILE)
        tok[st] |= (rng.integers(0, 3, int(st.sum())) << 4).astype(np.uint8)
        g = int(rng.integers(0, nv))
        ps = oracle_mod.check_program_guarded(tok, pay, nv, g)
        op = oracle_mod.check_program(np.where(st, tok & 15, tok).astype(np.uint8), pay, nv)
        assert np.all((ps[0] & ~op[0]) == 0)
        assert np.all((ps[1] & ~op[1]) == 0)
        assert ps[2] == -1 or (op[2] != -1 and ps[2] >= op[2])


def test_rejects_conditions_without_guard(oracle_mod):
    tok = np.array([IF | (1 << 4), NOOP, ELSE, NOOP, END], np.uint8)
    pay = np.array([1, 0, 1, 0, 0], np.int32)
    with pytest.raises(oracle_mod.OracleError):
        oracle_mod.check_program_guarded(tok, pay, 1, -1)
    with pytest.raises(oracle_mod.OracleError):
        oracle_mod.check_program_guarded(np.array([IF | (3 << 4), ELSE, END], np.uint8),
                                         np.array([0, 0, 0], np.int32), 1, 0)
