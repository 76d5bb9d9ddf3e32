"""Pins of the oracle's VectorPU mode over pvectors with lifetimes
(oracle_vectorpu_lifetimes).

References: Section 4.3 (r_v is updated at pvector creations and deletions
and queried at each call; the example of Section 4.3, with pvectors deleted or
created between its calls); Section 5's description of partial vectors (a new
pvector inherits the coherence state of its mother vector); the overlap
theorem of Section 4.2 on the live arrays, checked with a per-element model
written here (each element has its own validity pair, a vector's elements are
a fresh allocation when it is created, pvectors are windows onto them).  With
every array live throughout and no pvector, the mode reduces to the static
one (oracle_vectorpu), which keeps its overlap sets as a precomputed list
while this mode keeps r_v as an unordered list of live arrays.
"""
import json
import os

import numpy as np
import pytest

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")
R, W, RW, DROP = 1, 2, 3, 0x80
K_R, K_W, K_PUSH, K_PULL, K_NOOP, K_PW, K_GT, K_EN = range(8)
F = 4
II, VI, IV, VV = 0, 1, 2, 3


def leq(a, b):
    """The abstraction order of Section 3.3: (V,I) <= (V,V), (I,V) <= (V,V)."""
    return a == b or (b == VV and a in (VI, IV))


def csr(calls):
    side = np.array([c[0] for c in calls], np.uint8)
    off = np.zeros(len(calls) + 1, np.int32)
    arr, mode = [], []
    for i, c in enumerate(calls):
        for a, m in c[1]:
            arr.append(a)
            mode.append(m)
        off[i + 1] = len(arr)
    return side, off, np.array(arr, np.int32), np.array(mode, np.uint8)


def run(oracle_mod, arrays, calls, infer=True):
    """arrays: (start, len, parent, born, died) per array."""
    a = np.array(arrays, np.int64).reshape(-1, 5)
    side, off, arr, mode = csr(calls)
    return oracle_mod.vectorpu_lifetimes(a[:, 0], a[:, 1], a[:, 2], a[:, 3], a[:, 4], side, off, arr, mode,
                                         infer_overlap=infer)


def call_ops(res, c):
    a, b = res["call_first_op"][c], res["call_first_op"][c + 1]
    return res["kind_side"][a:b], res["var"][a:b], res["step_status"][a:b]


def random_static(rng, A, space, n_calls):
    starts = rng.integers(0, space - 8, A)
    lens = np.minimum(rng.integers(1, 40, A), space - starts)
    calls = []
    for _ in range(n_calls):
        k = int(rng.integers(1, min(4, A) + 1))
        ops = [(int(x), int(rng.choice([R, W, RW, R | DROP, W | DROP], p=[0.4, 0.25, 0.2, 0.1, 0.05])))
               for x in rng.choice(A, size=k, replace=False)]
        calls.append((int(rng.integers(0, 2)), ops))
    return [(int(s), int(l)) for s, l in zip(starts, lens)], calls


@pytest.mark.parametrize("infer", [True, False])
@pytest.mark.parametrize("seed", range(6))
def test_reduces_to_the_static_mode(oracle_mod, seed, infer):
    rng = np.random.default_rng(300 + seed)
    iv, calls = random_static(rng, 16, 160, 200)
    C = len(calls)
    side, off, arr, mode = csr(calls)
    s = np.array([x[0] for x in iv], np.int32)
    ln = np.array([x[1] for x in iv], np.int32)
    exp = oracle_mod.vectorpu(s, ln, side, off, arr, mode, infer_overlap=infer)
    got = run(oracle_mod, [(a, b, -1, 0, C) for a, b in iv], calls, infer=infer)
    for k in ("kind_side", "var", "step_status", "call_first_op", "final_status", "var_first_fault"):
        assert np.array_equal(exp[k], got[k]), k
    assert exp["first_fault"] == got["first_fault"]
    assert (got["arr_probe"] == -1).all()


def paper_example():
    g = json.load(open(os.path.join(GOLDEN, "section4_3_pvectors.json")))
    iv = [(a, b - a) for a, b in g["intervals"]]
    return iv, g["calls"]


def shadows_of(res, c, calls, A):
    ks, var, _ = call_ops(res, c)
    operands = {a for a, _ in calls[c][1]}
    guarded = {int(v) for k, v in zip(ks, var) if (k & 15) == K_GT}
    abs_written = {int(v) - A for k, v in zip(ks, var) if (k & 15) == K_W and v >= A}
    return sorted((guarded | abs_written) - operands)


def test_section4_3_example_live_throughout(oracle_mod):
    # pv1..pv4 created before f1 and never deleted: the paper's rewriting,
    # f2(W(pv3)) -> f2(W(pv3), RW(pv2))
    iv, calls = paper_example()
    res = run(oracle_mod, [(a, b, -1, 0, 3) for a, b in iv], calls)
    assert [shadows_of(res, c, calls, 4) for c in range(3)] == [[], [1], [0]]


def test_section4_3_example_with_deletion_and_late_creation(oracle_mod):
    # pv2 deleted after f1 (r_v loses it): f2 appends no RW(pv2) and writes
    # nothing of it, and f3 no longer names pv2; pv3 created only between f1
    # and f2; f3's RW(pv4) still shadows pv1, live throughout
    iv, calls = paper_example()
    calls = [calls[0], calls[1], (0, [(3, RW)])]
    arrays = [(iv[0][0], iv[0][1], -1, 0, 3), (iv[1][0], iv[1][1], -1, 0, 1),
              (iv[2][0], iv[2][1], -1, 1, 3), (iv[3][0], iv[3][1], -1, 0, 3)]
    calls[0] = (0, [(0, R), (1, R)])
    res = run(oracle_mod, arrays, calls)
    assert shadows_of(res, 1, calls, 4) == []
    ks, var, _ = call_ops(res, 1)
    assert not np.isin(var, [1, 4 + 1]).any()
    assert shadows_of(res, 2, calls, 4) == [0]


def test_mother_vector_is_in_the_overlap_relation(oracle_mod):
    # the same example with v = [0, 10) as an array and pv1..pv4 its pvectors:
    # v overlaps every pvector, so f2's W(pv3) shadows pv2 and v (the paper's
    # r_v lists only pvectors and leaves the whole vector to the programmer's
    # SX macros; kept in the relation, v's statuses stay sound for the
    # pvectors that inherit them)
    iv, calls = paper_example()
    arrays = [(a, b, 4, 0, 3) for a, b in iv] + [(0, 10, -1, 0, 3)]
    res = run(oracle_mod, arrays, calls)
    assert shadows_of(res, 1, calls, 5) == [1, 4]
    # every pvector was created before call 0 from v's initial statuses
    assert list(res["arr_probe"]) == [0, 2, 4, 6, -1]
    ks, var, st = call_ops(res, 0)
    assert list(ks[:8]) == [K_NOOP] * 8 and list(var[:8]) == [4, 9] * 4 and list(st[:8]) == [VI] * 8


def test_inherited_statuses_hand_derived(oracle_mod):
    # v = [0, 10) written on the GPU in call 0 (Fig. sem-AM: w v# then the
    # body's w v, both on the GPU side: (I,V)); pv = [2, 5) created before
    # call 1 inherits (I,V) for pv and pv#; call 1 reads pv on the CPU: the
    # guard finds pv# invalid on the CPU, so Pull pv; Pull pv# give (V,V), and
    # the read is fine
    arrays = [(0, 10, -1, 0, 2), (2, 3, 0, 1, 2)]
    calls = [(1, [(0, W)]), (0, [(1, R)])]
    res = run(oracle_mod, arrays, calls)
    A = 2
    ks, var, st = call_ops(res, 0)
    # w v#, w v; nothing of pv, which is not live yet (no shadow, no projection)
    assert list(ks) == [K_W | 16, K_W | 16] and list(var) == [A + 0, 0] and list(st) == [IV, IV]
    ks, var, st = call_ops(res, 1)
    assert list(ks) == [K_NOOP, K_NOOP, K_GT, K_EN, K_R]
    assert list(var) == [0, A + 0, 1, A + 1, 1]
    assert list(st) == [IV, IV, VV, VV, VV]
    assert res["arr_probe"][1] == res["call_first_op"][1] and res["arr_probe"][0] == -1
    assert res["first_fault"] == -1


@pytest.mark.parametrize("bad", [
    [(0, 10, -1, 0, 2), (2, 3, 0, 0, 2)],       # fine (control)
    [(0, 10, -1, 1, 2), (2, 3, 0, 0, 2)],       # pvector born before its vector
    [(0, 10, -1, 0, 1), (2, 3, 0, 0, 2)],       # pvector outliving its vector
    [(0, 10, -1, 0, 2), (8, 3, 0, 0, 2)],       # range not inside the vector's
    [(0, 10, 1, 0, 2), (2, 3, 0, 0, 2)],        # a pvector's pvector
    [(0, 10, -1, 0, 2), (2, 3, 1, 0, 2)],       # its own vector
    [(0, 10, -1, 1, 1), (2, 3, 0, 1, 2)],       # empty lifetime
    [(0, 10, -1, 0, 3), (2, 3, 0, 0, 2)],       # died after the last call
])
def test_rejects_malformed_lifetimes(oracle_mod, bad):
    calls = [(0, [(0, R)]), (0, [(0, R)])]
    if bad == [(0, 10, -1, 0, 2), (2, 3, 0, 0, 2)]:
        run(oracle_mod, bad, calls)
        return
    with pytest.raises(oracle_mod.OracleError):
        run(oracle_mod, bad, calls)


def test_rejects_dead_operands(oracle_mod):
    arrays = [(0, 10, -1, 0, 2), (2, 3, 0, 1, 2)]
    with pytest.raises(oracle_mod.OracleError):
        run(oracle_mod, arrays, [(0, [(1, R)]), (0, [(0, R)])])


# --------------------------------------------------------------------------
# Per-element model with lifetimes
# --------------------------------------------------------------------------
def random_lifetimes(rng, n_vectors=2, n_pvectors=12, vec_len=64, n_calls=150, late_vector=True,
                     modes=(R, W, RW), p=(0.5, 0.3, 0.2), drop_p=0.0):
    arrays = []
    for v in range(n_vectors):
        born = int(rng.integers(1, n_calls // 3)) if (late_vector and v == n_vectors - 1) else 0
        arrays.append((v * vec_len, vec_len, -1, born, n_calls))
    for _ in range(n_pvectors):
        v = int(rng.integers(0, n_vectors))
        s = int(rng.integers(0, vec_len - 1))
        ln = int(rng.integers(1, vec_len - s + 1))
        born = int(rng.integers(arrays[v][3], n_calls - 1))
        died = int(rng.integers(born + 1, n_calls + 1))
        arrays.append((v * vec_len + s, ln, v, born, died))
    calls = []
    for c in range(n_calls):
        live = [a for a, x in enumerate(arrays) if x[3] <= c < x[4]]
        k = int(rng.integers(1, min(3, len(live)) + 1))
        ops = []
        for a in rng.choice(live, size=k, replace=False):
            m = int(rng.choice(modes, p=p))
            if rng.random() < drop_p:
                m |= DROP
            ops.append((int(a), m))
        calls.append((int(rng.integers(0, 2)), ops))
    return arrays, calls


class ElementModel:
    def __init__(self, arrays, space):
        self.arrays = arrays
        self.elem = np.full(space, VI, np.int64)
        self.abs = [VI] * len(arrays)
        self.faults = 0

    def rng(self, a):
        s, ln = self.arrays[a][0], self.arrays[a][1]
        return slice(s, s + ln)

    def live(self, a, c):
        return self.arrays[a][3] <= c < self.arrays[a][4]

    def ov(self, a, b):
        (s1, l1), (s2, l2) = self.arrays[a][:2], self.arrays[b][:2]
        return s1 < s2 + l2 and s2 < s1 + l1

    def create(self, c):
        for a, x in enumerate(self.arrays):
            if x[3] != c:
                continue
            if x[2] < 0:
                self.elem[self.rng(a)] = VI          # a fresh allocation
                self.abs[a] = VI
            else:
                self.abs[a] = self.abs[x[2]]         # inherited from the mother vector

    def om(self, c, call):
        side, ops = call
        declared = {a: m for a, m in ops if not (m & DROP)}
        args = {a for a, _ in ops}
        eff = dict(declared)
        shadows = set()
        for x, mx in declared.items():
            if mx not in (W, RW):
                continue
            for y in range(len(self.arrays)):
                if y == x or not self.live(y, c) or not self.ov(x, y):
                    continue
                if y in declared:
                    if mx == RW or declared[y] != W:
                        eff[y] = RW
                elif y not in args:
                    shadows.add(y)
        return eff, sorted(shadows)

    def step(self, c, call, infer=True):
        self.create(c)
        side, ops = call
        eff, shadows = self.om(c, call) if infer else ({a: m for a, m in ops if not m & DROP}, [])
        for a, me in [(a, eff[a]) for a, m in ops if not (m & DROP)] + [(y, RW) for y in shadows]:
            if me in (R, RW) and not ((self.abs[a] >> side) & 1):
                e = self.elem[self.rng(a)]
                if np.any(((e >> (1 - side)) & 1) == 0):
                    self.faults += 1
                self.elem[self.rng(a)] = VV
                self.abs[a] = VV
            if me in (W, RW):
                self.abs[a] = VI if side == 0 else IV
        for a, m in ops:
            if (m & 3) in (R, RW) and np.any(((self.elem[self.rng(a)] >> side) & 1) == 0):
                self.faults += 1
            if (m & 3) in (W, RW):
                self.elem[self.rng(a)] = VI if side == 0 else IV


def summaries(res, arrays, n_calls):
    """Statuses of all 2A variables after each call, from the step outputs and
    the creation records."""
    A = len(arrays)
    st = np.full(2 * A, VI, np.int64)
    probe_of = {int(p): a for a, p in enumerate(res["arr_probe"]) if p >= 0}
    out = []
    for c in range(n_calls):
        for a, x in enumerate(arrays):
            if x[2] < 0 and x[3] == c:
                st[a] = st[A + a] = VI
        lo, hi = res["call_first_op"][c], res["call_first_op"][c + 1]
        for j in range(lo, hi):
            st[res["var"][j]] = res["step_status"][j]
            if j in probe_of:
                a = probe_of[j]
                st[a], st[A + a] = res["step_status"][j], res["step_status"][j + 1]
        out.append(st.copy())
    return out


@pytest.mark.parametrize("seed", range(16))
def test_overlap_theorem_with_lifetimes(oracle_mod, seed):
    """Section 4.2's theorem on the live arrays at every call: the element
    model never faults and keeps sigma(x#) <= sigma(x[i]) for every live x;
    the oracle never faults, its abstract statuses equal the model's, and a
    side it calls valid is valid for every element of a live array."""
    rng = np.random.default_rng(700 + seed)
    arrays, calls = random_lifetimes(rng)
    res = run(oracle_mod, arrays, calls)
    summ = summaries(res, arrays, len(calls))
    m = ElementModel(arrays, 2 * 64)
    A = len(arrays)
    for c, call in enumerate(calls):
        m.step(c, call)
        st = summ[c]
        for x in range(A):
            if not m.live(x, c):
                continue
            e = m.elem[m.rng(x)]
            assert m.abs[x] == st[A + x], (c, x)
            assert all(leq(m.abs[x], int(s)) for s in e), (c, x)
            if st[x] != F:
                for side in (0, 1):
                    if (st[x] >> side) & 1:
                        assert np.all((e >> side) & 1), (c, x, side)
    assert m.faults == 0
    assert res["first_fault"] == -1


def test_inherited_statuses_are_not_always_the_initial_store(oracle_mod):
    # over the random programs, pvectors are often created from a vector whose
    # statuses are no longer (V,I): inheritance is exercised
    found = 0
    for seed in range(10):
        rng = np.random.default_rng(700 + seed)
        arrays, calls = random_lifetimes(rng)
        res = run(oracle_mod, arrays, calls)
        for a, p in enumerate(res["arr_probe"]):
            if p >= 0 and (res["step_status"][p] != VI or res["step_status"][p + 1] != VI):
                found += 1
    assert found >= 10


def test_inheritance_has_teeth(oracle_mod):
    """Giving every pvector the initial store's (V,I) at its creation instead
    of its vector's statuses is unsound: on some programs a side the summary
    calls valid is invalid for an element."""
    unsound = 0
    for seed in range(20):
        rng = np.random.default_rng(900 + seed)
        arrays, calls = random_lifetimes(rng, late_vector=False)
        fresh = [(s, ln, -1, b, d) for s, ln, p, b, d in arrays]      # no inheritance
        res = run(oracle_mod, fresh, calls)
        summ = summaries(res, fresh, len(calls))
        m = ElementModel(arrays, 2 * 64)
        bad = False
        for c, call in enumerate(calls):
            m.step(c, call)
            st = summ[c]
            for x in range(len(arrays)):
                if not m.live(x, c) or st[x] == F:
                    continue
                e = m.elem[m.rng(x)]
                for side in (0, 1):
                    if (st[x] >> side) & 1 and not np.all((e >> side) & 1):
                        bad = True
        unsound += bad
    assert unsound >= 3


def test_abstract_variables_never_invalid_nor_stuck(oracle_mod):
    # Property Safety on the abstract variables carries over: inheritance copies
    # a vector's abstract status, which is never (I,I) or F
    rng = np.random.default_rng(950)
    for _ in range(10):
        arrays, calls = random_lifetimes(rng, drop_p=0.2)
        res = run(oracle_mod, arrays, calls)
        A = len(arrays)
        abstract = res["var"] >= A
        assert not np.isin(res["step_status"][abstract], [II, F]).any()
        assert not np.isin(res["final_status"][A:], [II, F]).any()
