"""Serving: continuous batching with device-resident session statuses.

Each request's result is the same when it runs alone (one slot, requests
submitted one at a time) and in the mix (many slots, all sessions submitted
at once, their work overlapping on the GPU), and both equal the oracle run of
the session's requests in order (the session's final statuses of one request
are the initial statuses of the next)."""
import time

import numpy as np
import pytest

import workloads

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def amc():
    import paper_1910_11110_gb300 as m
    m.build()
    return m


def make_sessions(seed=7, n_sessions=12):
    rng = np.random.default_rng(seed)
    sessions = []
    for s in range(n_sessions):
        nv = int(rng.integers(8, 300))
        kind = s % 2                      # sessions are typed by their first request
        reqs = []
        for r in range(int(rng.integers(1, 7))):
            if kind == 0:
                n = int(2 ** rng.uniform(3, 17))
                ks, var = workloads.trace_random(rng, n, nv, p=[0.3, 0.35, 0.1, 0.1, 0.15])
                reqs.append((ks, var))
            else:
                b = workloads.programs(1, seed=1000 + s, first=r, median=300.0, max_len=3000,
                                       vars_lo=nv, vars_hi=nv)
                reqs.append((b["tok"], b["payload"]))
        sessions.append((s, kind, nv, reqs))
    return sessions


def oracle_results(oracle_mod, sessions):
    out = {}
    for sid, kind, nv, reqs in sessions:
        st = None
        for i, (a, b) in enumerate(reqs):
            if kind == 0:
                step, st, vff, ff = oracle_mod.check_trace(a, b, nv, init_status=st)
                out[(sid, i)] = (step, ff)
            else:
                step, st, ff = oracle_mod.check_program(a, b, nv, init_mask=st)
                out[(sid, i)] = (step, ff)
    return out


def run_server(amc, sessions, slots, one_at_a_time):
    res = {}
    with amc.Server(mem_budget_bytes=1 << 30, max_slots=slots) as srv:
        pending = {}
        order = [(sid, kind, nv, i, r) for sid, kind, nv, reqs in sessions for i, r in enumerate(reqs)]
        if not one_at_a_time:      # interleave sessions: round robin by request index
            order.sort(key=lambda x: (x[3], x[0]))
        for sid, kind, nv, i, (a, b) in order:
            t = srv.submit(sid, kind, nv, a, b)
            assert t is not None
            pending[t] = (sid, i)
            if one_at_a_time:
                while (r := srv.poll(t)) is None:
                    time.sleep(1e-4)
                res[(sid, i)] = r
                del pending[t]
        deadline = time.time() + 120
        while pending and time.time() < deadline:
            for t in list(pending):
                r = srv.poll(t)
                if r is not None:
                    res[pending.pop(t)] = r
            time.sleep(1e-4)
        assert not pending
        finals = {sid: srv.export(sid, nv) for sid, kind, nv, _ in sessions}
    return res, finals


def test_alone_equals_mix_equals_oracle(amc, oracle_mod):
    sessions = make_sessions()
    exp = oracle_results(oracle_mod, sessions)
    alone, fin_a = run_server(amc, sessions, slots=1, one_at_a_time=True)
    mix, fin_m = run_server(amc, sessions, slots=16, one_at_a_time=False)
    for key, (step, ff) in exp.items():
        for got in (alone[key], mix[key]):
            assert got["error"] == 0
            assert np.array_equal(got["status"], step), key
            assert got["first_fault"] == ff, key
    for sid in fin_a:
        assert np.array_equal(fin_a[sid], fin_m[sid])


def test_rejects_malformed_requests(amc):
    with amc.Server(mem_budget_bytes=1 << 26, max_slots=2) as srv:
        with pytest.raises(amc.AmcError):
            srv.submit(1, 0, 4, np.array([0, 1], np.uint8), np.array([0, 9], np.int32))
        with pytest.raises(amc.AmcError):
            srv.submit(2, 1, 4, np.array([8, 0], np.uint8), np.array([1, 0], np.int32))
        t = srv.submit(3, 0, 4, np.array([1, 4], np.uint8), np.array([0, 0], np.int32))
        while (r := srv.poll(t)) is None:
            time.sleep(1e-4)
        assert r["status"].tolist() == [1, 1] and r["first_fault"] == -1
        with pytest.raises(amc.AmcError):           # a trace session cannot take a program
            srv.submit(3, 1, 4, np.array([0], np.uint8), np.array([0], np.int32))
