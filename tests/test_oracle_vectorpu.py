"""Pins of the oracle's VectorPU mode (translation of access modes, overlap
inference, per-array statuses).

References: the worked examples of Sections 3.4 and 4.3; the VectorPU flag
code of Fig. vectorpucoherence (an independent formulation of the same
protocol, Section 3.6); Theorems Subject reduction and Progress for
well-declared programs (Section 3.4), their array versions (Section 3.5) and
the overlap theorem of Section 4.2, checked with a per-element array model
written here from Section 3.5 (each element has its own validity pair,
overlapping arrays share elements, Push/Pull move whole arrays).
"""
import json
import os

import numpy as np
import pytest

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")
R, W, RW, DROP = 1, 2, 3, 0x80
K_R, K_W, K_PUSH, K_PULL, K_NOOP, K_PW, K_GT, K_EN = range(8)
F = 4
VI, IV, VV, II = 1, 2, 3, 0


def leq(a, b):
    """The abstraction order of Section 3.3: (V,I) <= (V,V), (I,V) <= (V,V),
    reflexive."""
    return a == b or (b == VV and a in (VI, IV))


def calls_to_csr(calls):
    side = np.array([c[0] for c in calls], np.uint8)
    off = np.zeros(len(calls) + 1, np.int32)
    arr, mode = [], []
    for i, c in enumerate(calls):
        for a, m in c[1]:
            arr.append(a)
            mode.append(m)
        off[i + 1] = len(arr)
    return side, off, np.array(arr, np.int32), np.array(mode, np.uint8)


def run(oracle_mod, intervals, calls, infer=True):
    s = np.array([iv[0] for iv in intervals], np.int32)
    ln = np.array([iv[1] for iv in intervals], np.int32)
    side, off, arr, mode = calls_to_csr(calls)
    return oracle_mod.vectorpu(s, ln, side, off, arr, mode, infer_overlap=infer)


def call_slots(res, c):
    a, b = res["call_first_op"][c], res["call_first_op"][c + 1]
    return res["kind_side"][a:b], res["var"][a:b], res["step_status"][a:b]


def test_section3_4_example(oracle_mod):
    g = json.load(open(os.path.join(GOLDEN, "section3_4_example.json")))
    res = run(oracle_mod, g["arrays"], g["calls"])
    A = len(g["arrays"])
    ks, var, st = call_slots(res, 0)
    # after the first block the abstract variable is (V,I)
    assert st[var == A].tolist()[-1] == g["abstract_after_first_call"]
    ks, var, st = call_slots(res, 1)
    # the GPU-side read guard fails, so Push x; Push x# run: both become (V,V)
    gt = np.nonzero((ks & 15) == K_GT)[0]
    assert len(gt) == 1 and var[gt[0]] == 0 and (ks[gt[0]] >> 4) == 1
    assert st[gt[0]] == VV and st[gt[0] + 1] == VV
    assert g["second_call_transfers"]
    assert res["first_fault"] == -1 and g["faults"] == 0


@pytest.mark.parametrize("inclusive", [True, False])
def test_section4_3_pvectors(oracle_mod, inclusive):
    g = json.load(open(os.path.join(GOLDEN, "section4_3_pvectors.json")))
    if inclusive:
        iv = [(a, b - a + 1) for a, b in g["intervals"]]
    else:
        iv = [(a, b - a) for a, b in g["intervals"]]
    res = run(oracle_mod, iv, g["calls"])
    A = len(iv)
    for c, call in enumerate(g["calls"]):
        ks, var, st = call_slots(res, c)
        operands = {a for a, _ in call[1]}
        guarded = {int(v) for k, v in zip(ks, var) if (k & 15) == K_GT}
        abs_written = {int(v) - A for k, v in zip(ks, var) if (k & 15) == K_W and v >= A}
        shadows = sorted((guarded | abs_written) - operands)
        assert shadows == g["shadows"][c], (c, shadows)
    assert res["first_fault"] == -1


def flag_code(mode, side, cpu_flag, gpu_flag):
    """Fig. vectorpucoherence: coherent_on_{cpu,gpu}_{r,w,rw}.  Returns the new
    flags and whether a download/upload was performed."""
    moved = False
    if side == 0:
        if mode in (R, RW):
            if not cpu_flag:
                moved = True
                cpu_flag = True
            if mode == RW:
                gpu_flag = False
        else:
            cpu_flag, gpu_flag = True, False
    else:
        if mode in (R, RW):
            if not gpu_flag:
                moved = True
                gpu_flag = True
            if mode == RW:
                cpu_flag = False
        else:
            gpu_flag, cpu_flag = True, False
    return cpu_flag, gpu_flag, moved


# call prefixes that drive the abstract status of array 0 to (V,I), (I,V), (V,V)
PREFIX = {VI: [], IV: [(1, [(0, W)])], VV: [(0, [(0, R)]), (1, [(0, R)])]}


@pytest.mark.parametrize("mode", [R, W, RW])
@pytest.mark.parametrize("side", [0, 1])
@pytest.mark.parametrize("start", [VI, IV, VV])
def test_translation_matches_flag_code(oracle_mod, mode, side, start):
    calls = PREFIX[start] + [(side, [(0, mode)])]
    res = run(oracle_mod, [(0, 64)], calls)
    c = len(calls) - 1
    pre_ks, pre_var, pre_st = (res["kind_side"][:res["call_first_op"][c]], res["var"][:res["call_first_op"][c]],
                               res["step_status"][:res["call_first_op"][c]])
    before = pre_st[pre_var == 1][-1] if np.any(pre_var == 1) else VI
    assert before == start
    ks, var, st = call_slots(res, c)
    after = st[var == 1][-1]
    moved = bool(np.any(((ks & 15) == K_EN) & (st != before)))
    cpu_f, gpu_f, exp_moved = flag_code(mode, side, bool(start & 1), bool(start & 2))
    assert after == (int(cpu_f) | int(gpu_f) << 1)
    assert moved == exp_moved
    assert res["first_fault"] == -1


def test_emitted_trace_replays_in_trace_mode(oracle_mod):
    import workloads
    w = workloads.vectorpu_calls(seed=21, n_arrays=64, space=1 << 14, n_calls=3000,
                                 len_log2=(4.0, 10.0), drop_p=0.02)
    res = oracle_mod.vectorpu(**w)
    A = len(w["arr_start"])
    step, final, vff, ff = oracle_mod.check_trace(res["kind_side"], res["var"], 2 * A)
    assert np.array_equal(step, res["step_status"])
    assert np.array_equal(final, res["final_status"])
    assert np.array_equal(vff, res["var_first_fault"])
    assert ff == res["first_fault"]


# --------------------------------------------------------------------------
# Per-element model (Section 3.5): the reference the summary is checked against
# --------------------------------------------------------------------------
def requires(kind, side, s):
    """True when the element access is possible (Property Progress)."""
    own = (s >> side) & 1
    other = (s >> (1 - side)) & 1
    if kind == K_R:
        return bool(own)
    return True


class ElementModel:
    """Elements of one shared index space, each with its own validity pair;
    an array is a range of elements.  Abstract statuses per array."""

    def __init__(self, intervals, space):
        self.iv = intervals
        self.elem = np.full(space, VI, np.int64)
        self.abs = [VI] * len(intervals)
        self.faults = 0

    def rng(self, a):
        s, l = self.iv[a]
        return slice(s, s + l)

    def transfer(self, a, side):
        # CPU-side declarations emit Pull (needs the GPU copy), GPU-side ones Push
        e = self.elem[self.rng(a)]
        need = 2 if side == 0 else 1
        if np.any((e & need) == 0):
            self.faults += 1
        self.elem[self.rng(a)] = VV

    def read(self, a, side):
        e = self.elem[self.rng(a)]
        if np.any(((e >> side) & 1) == 0):
            self.faults += 1

    def write(self, a, side):
        self.elem[self.rng(a)] = VI if side == 0 else IV


def om_decisions(intervals, call):
    """O(M) from Table Overlap-ext-tab, written out here: effective declared
    modes and the shadow set."""
    side, ops = call
    declared = {a: m for a, m in ops if not (m & DROP)}
    args = {a for a, _ in ops}
    eff = dict(declared)
    shadows = set()

    def ov(a, b):
        (s1, l1), (s2, l2) = intervals[a], intervals[b]
        return s1 < s2 + l2 and s2 < s1 + l1

    for x, mx in declared.items():
        if mx not in (W, RW):
            continue
        for y in range(len(intervals)):
            if y == x or not ov(x, y):
                continue
            if y in declared:
                if mx == RW or declared[y] != W:
                    eff[y] = RW
            elif y not in args:
                shadows.add(y)
    return eff, sorted(shadows)


def element_run(intervals, space, calls, infer=True, check=None):
    m = ElementModel(intervals, space)
    flip = lambda s, side: ((s >> side) & 1)
    for ci, call in enumerate(calls):
        side, ops = call
        eff, shadows = om_decisions(intervals, call) if infer else ({a: mm for a, mm in ops if not mm & DROP}, [])
        entries = [(a, eff[a]) for a, mm in ops if not (mm & DROP)] + [(y, RW) for y in shadows]
        for a, me in entries:
            if me in (R, RW) and not flip(m.abs[a], side):
                m.transfer(a, side)
                m.abs[a] = VV if m.abs[a] != II else F
            if me in (W, RW):
                m.abs[a] = VI if side == 0 else IV
        for a, mm in ops:
            mo = mm & 3
            if mo in (R, RW):
                m.read(a, side)
            if mo in (W, RW):
                m.write(a, side)
        if check:
            check(ci, m)
    return m


def random_calls(rng, n_arrays, n_calls, drop_p=0.0, modes=(R, W, RW), p=(0.5, 0.3, 0.2)):
    calls = []
    for _ in range(n_calls):
        k = int(rng.integers(1, min(4, n_arrays) + 1))
        arrs = rng.choice(n_arrays, size=k, replace=False)
        ops = []
        for a in arrs:
            mm = int(rng.choice(modes, p=p))
            if rng.random() < drop_p:
                mm |= DROP
            ops.append((int(a), mm))
        calls.append((int(rng.integers(0, 2)), ops))
    return calls


def summary_per_call(res, n_calls, A):
    """Statuses of all 2A variables after each call, from the step outputs."""
    st = np.full(2 * A, VI, np.int64)
    out = []
    for c in range(n_calls):
        a, b = res["call_first_op"][c], res["call_first_op"][c + 1]
        for j in range(a, b):
            st[res["var"][j]] = res["step_status"][j]
        out.append(st.copy())
    return out


@pytest.mark.parametrize("seed", range(12))
def test_theorems_disjoint_arrays(oracle_mod, seed):
    """Subject reduction + Progress for well-declared programs (Sections 3.4,
    3.5): no fault, and sigma(x#) <= sigma(x) after every call."""
    rng = np.random.default_rng(seed)
    A = 12
    intervals = [(64 * a, 64) for a in range(A)]
    calls = random_calls(rng, A, 300)
    res = run(oracle_mod, intervals, calls)
    assert res["first_fault"] == -1
    for st in summary_per_call(res, len(calls), A):
        for x in range(A):
            assert leq(st[A + x], st[x])


@pytest.mark.parametrize("seed", range(16))
def test_overlap_theorem_element_model(oracle_mod, seed):
    """Section 4.2 theorem with O(M): the element model never faults and keeps
    sigma(x#) <= sigma(x[i]); the oracle's per-array summary never faults, its
    abstract statuses equal the element model's, and the summary is sound:
    a side it calls valid is valid for every element."""
    rng = np.random.default_rng(100 + seed)
    A, space = 10, 96
    starts = rng.integers(0, space - 8, A)
    lens = rng.integers(1, 40, A)
    lens = np.minimum(lens, space - starts)
    intervals = [(int(s), int(l)) for s, l in zip(starts, lens)]
    calls = random_calls(rng, A, 150)
    res = run(oracle_mod, intervals, calls)
    summ = summary_per_call(res, len(calls), A)

    def check(ci, m):
        st = summ[ci]
        for x in range(A):
            e = m.elem[m.rng(x)]
            assert m.abs[x] == st[A + x]
            for s in e:
                assert leq(m.abs[x], int(s)), (ci, x)
            if st[x] != F:
                for side in (0, 1):
                    if (st[x] >> side) & 1:
                        assert np.all((e >> side) & 1), (ci, x, side)

    m = element_run(intervals, space, calls, check=check)
    assert m.faults == 0
    assert res["first_fault"] == -1


def test_overlap_inference_has_teeth(oracle_mod):
    """Without O(M) random overlapping programs do access invalid elements."""
    found = 0
    for seed in range(20):
        rng = np.random.default_rng(500 + seed)
        A, space = 8, 64
        starts = rng.integers(0, space - 8, A)
        lens = np.minimum(rng.integers(4, 40, A), space - starts)
        intervals = [(int(s), int(l)) for s, l in zip(starts, lens)]
        calls = random_calls(rng, A, 100)
        m = element_run(intervals, space, calls, infer=False)
        res = run(oracle_mod, intervals, calls, infer=False)
        found += m.faults > 0
        if m.faults > 0:
            assert res["first_fault"] >= 0     # the sound summary reports it too
    assert found >= 5


def test_section3_5_partial_write_example():
    """Section 3.5 example: a GPU write of x[3] alone is only safe under
    rem(RW x#); under rem(W x#) the abstraction stops being correct."""
    iv = [(0, 8)]
    # rem(W x#) { rem(w x[3]) }
    m = ElementModel(iv, 8)
    m.abs[0] = IV                       # [[rem(W x#)]] = rem(w x#)
    m.elem[3] = IV                      # rem(w x[3])
    assert not all(leq(m.abs[0], int(s)) for s in m.elem)
    # rem(RW x#) { rem(w x[3]) }: remIsValid x# fails, Push x; Push x#; rem(w x#)
    m = ElementModel(iv, 8)
    m.transfer(0, 1)
    m.abs[0] = IV
    m.elem[3] = IV
    assert m.faults == 0 and all(leq(m.abs[0], int(s)) for s in m.elem)


def test_dropped_annotations_can_fault(oracle_mod):
    rng = np.random.default_rng(77)
    A = 6
    intervals = [(32 * a, 32) for a in range(A)]
    hits = 0
    for _ in range(10):
        calls = random_calls(rng, A, 200, drop_p=0.2)
        res = run(oracle_mod, intervals, calls)
        m = element_run(intervals, 32 * A, calls)
        hits += res["first_fault"] >= 0
        assert (res["first_fault"] >= 0) == (m.faults > 0)   # disjoint: summary is exact
    assert hits >= 3


def test_rejects_duplicate_operands(oracle_mod):
    with pytest.raises(oracle_mod.OracleError):
        run(oracle_mod, [(0, 4), (4, 4)], [(0, [(0, R), (0, W)])])


@pytest.mark.parametrize("infer", [True, False])
def test_abstract_variables_never_invalid_nor_stuck(oracle_mod, infer):
    # Property Safety carried to the abstract variables of Section 3.5: only
    # w x#, and the Pull / Push of a guard that found its side invalid, act on
    # x#; w gives (V,I) or (I,V), and the guard's transfer runs only when the
    # side is invalid, which from (V,I) / (I,V) / (V,V) means the other side
    # is valid.  So no abstract variable reaches (I,I), and EN never gives F,
    # with or without O(M) and whatever annotations are dropped (dropped ones
    # add body accesses on real arrays only).  Overlapping arrays, drops at
    # one in five.
    rng = np.random.default_rng(81 if infer else 82)
    A = 8
    intervals = [(int(rng.integers(0, 200)), int(rng.integers(1, 80))) for _ in range(A)]
    n_en = 0
    for _ in range(20):
        calls = random_calls(rng, A, 150, drop_p=0.2)
        res = run(oracle_mod, intervals, calls, infer=infer)
        abstract = res["var"] >= A
        st = res["step_status"][abstract]
        assert not np.isin(st, [II, F]).any()
        en = (res["kind_side"] & 15) == K_EN
        n_en += int(en.sum())
        assert not (res["step_status"][en] == F).any()
        assert not np.isin(res["final_status"][A:], [II, F]).any()
    assert n_en > 100
