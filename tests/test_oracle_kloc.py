"""The oracle's check over k memory locations (the Section 3.1 signatures on
a vector of k validity flags; Section 3 and the conclusion state that the
two-location results extend to many locations).  Pinned by the two-location
calculus it must reduce to, by its projection onto any two locations a trace
uses, by relabelling locations, and by Property Safety and Property Progress
carried to k locations."""
import numpy as np
import pytest

import workloads

KL_F = 0x80


def kop(kind, a=0, b=0):
    return kind | a << 2 | b << 5


# two-location op byte (kind | side << 4) -> k-location op byte, local = 0
def embed2(ks):
    kind, side = ks & 15, ks >> 4
    if kind == 0:
        return kop(0, side)
    if kind == 1:
        return kop(1, side)
    if kind == 2:                       # Push: upload the op's own location into the other
        return kop(2, side, 1 - side)
    if kind == 3:                       # Pull: download the other location into the op's own
        return kop(2, 1 - side, side)
    return kop(3)


def random_kloc(rng, n, n_vars, k, p_copy=0.3):
    kind = rng.choice(4, size=n, p=[0.35, 0.2, p_copy, 0.15 - (p_copy - 0.3)])
    a = rng.integers(0, k, n)
    b = (a + rng.integers(1, k, n)) % k if k > 1 else a
    op = np.where(kind == 3, 3, np.where(kind == 2, kind | a << 2 | b << 5, kind | a << 2)).astype(np.uint8)
    if k == 1:
        op[kind == 2] = 3
    return op, rng.integers(0, n_vars, n).astype(np.int32)


def test_reduces_to_two_locations(oracle_mod):
    # k = 2: every output equals the two-location check's (status codes
    # cpuValid | gpuValid << 1 are the same bit masks; F = 4 <-> 0x80)
    rng = np.random.default_rng(61)
    for _ in range(4):
        ks, var = workloads.trace_random(rng, 20_000, 300)
        init = rng.integers(0, 5, 300).astype(np.uint8)
        e = oracle_mod.check_trace(ks, var, 300, init)
        op = np.array([embed2(int(x)) for x in ks], np.uint8)
        g = oracle_mod.check_trace_k(op, var, 300, 2, np.where(init == 4, KL_F, init).astype(np.uint8))
        m = lambda s: np.where(s == KL_F, 4, s)
        assert np.array_equal(e[0], m(g[0])) and np.array_equal(e[1], m(g[1]))
        assert np.array_equal(e[2], g[2]) and e[3] == g[3]


@pytest.mark.parametrize("k", [3, 5, 7])
def test_projection_on_two_locations(oracle_mod, k):
    # a trace whose ops use only locations i and j: those two flags follow the
    # two-location check with i local and j remote
    rng = np.random.default_rng(62 + k)
    i, j = 1, k - 1
    ks, var = workloads.trace_random(rng, 20_000, 200)
    op2 = np.array([embed2(int(x)) for x in ks], np.uint8)
    remap = lambda loc: np.where(loc == 0, i, j)
    kind, a, b = op2 & 3, (op2 >> 2) & 7, (op2 >> 5) & 7
    op = np.where(kind == 3, 3, kind | remap(a) << 2 | np.where(kind == 2, remap(b), 0) << 5).astype(np.uint8)
    init = np.full(200, 1 << i, np.uint8)
    g = oracle_mod.check_trace_k(op, var, 200, k, init)
    e = oracle_mod.check_trace(ks, var, 200)
    proj = lambda s: np.where(s == KL_F, 4, ((s >> i) & 1) | ((s >> j) & 1) << 1)
    assert np.array_equal(proj(g[0]), e[0]) and np.array_equal(proj(g[1]), e[1]) and g[3] == e[3]
    # the flags of the other locations stay I
    live = g[0] != KL_F
    others = np.bitwise_and(g[0][live], 0x7F & ~((1 << i) | (1 << j)))
    assert not others.any()


def test_relabelling_locations(oracle_mod):
    # a permutation of the location ids applied to ops and initial statuses
    # permutes every status the same way
    rng = np.random.default_rng(63)
    k = 5
    op, var = random_kloc(rng, 30_000, 400, k)
    init = rng.integers(1, 1 << k, 400).astype(np.uint8)
    perm = rng.permutation(k)
    pm = lambda s: np.where(s == KL_F, KL_F, sum(((s >> t) & 1) << perm[t] for t in range(k))).astype(np.uint8)
    kind, a, b = op & 3, (op >> 2) & 7, (op >> 5) & 7
    op_p = np.where(kind == 3, 3, kind | perm[a] << 2 | np.where(kind == 2, perm[b], 0) << 5).astype(np.uint8)
    e = oracle_mod.check_trace_k(op, var, 400, k, init)
    g = oracle_mod.check_trace_k(op_p, var, 400, k, pm(init))
    assert np.array_equal(pm(e[0]), g[0]) and np.array_equal(pm(e[1]), g[1]) and e[3] == g[3]


@pytest.mark.parametrize("k", [1, 2, 4, 7])
def test_safety_and_progress(oracle_mod, k):
    # Safety: from "valid in location 0 only", no variable ever has no valid
    # location; Progress: an op is stuck exactly when the location it reads
    # (r at a, copy from a) is invalid before it
    rng = np.random.default_rng(64 + k)
    op, var = random_kloc(rng, 30_000, 100, k)
    step, final, vff, ff = oracle_mod.check_trace_k(op, var, 100, k)
    assert not (step == 0).any()
    prev = np.full(100, 1, np.int64)
    for x, v, s in zip(op.tolist(), var.tolist(), step.tolist()):
        kind, a = x & 3, (x >> 2) & 7
        if prev[v] != KL_F and kind in (0, 2):
            assert (s == KL_F) == (not (prev[v] >> a) & 1)
        prev[v] = s


def test_rejects_malformed(oracle_mod):
    z = np.zeros(1, np.int32)
    for bad, k in ((kop(2, 1, 1), 3), (kop(0, 3), 3), (kop(3, 1), 3), (kop(0, 0, 2), 3), (kop(0), 8)):
        with pytest.raises(oracle_mod.OracleError):
            oracle_mod.check_trace_k(np.array([bad], np.uint8), z, 1, k)
