"""Serving: continuous batching with device-resident session statuses.

Each request's result is the same when it runs alone (one slot, requests
submitted one at a time) and in the mix (many slots, all sessions submitted
at once, their work overlapping on the GPU), and both equal the oracle run of
the session's requests in order (the session's final statuses of one request
are the initial statuses of the next); so do the sessions' final status sets.
Sessions mix trace and program requests."""
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
    """Sessions whose requests are traces or programs, drawn per request.
    Sessions s % 3 == 0 start with a program holding If / While, so that their
    later traces see sets of several statuses; sessions s % 3 == 1 mix traces
    with straight-line programs (every set stays a singleton); sessions
    s % 3 == 2 mix traces with programs holding If / While."""
    rng = np.random.default_rng(seed)
    sessions = []
    for s in range(n_sessions):
        nv = int(rng.integers(8, 300))
        reqs = []
        for r in range(int(rng.integers(2, 7))):
            if (s % 3 == 0 and r == 0) or rng.random() < 0.4:
                p = (0.0, 0.0) if s % 3 == 1 else (0.2, 0.1)
                b = workloads.programs(1, seed=1000 + s, first=r, median=300.0, max_len=3000,
                                       vars_lo=nv, vars_hi=nv, p_if=p[0], p_while=p[1])
                reqs.append((1, b["tok"], b["payload"]))
            else:
                n = int(2 ** rng.uniform(3, 17))
                ks, var = workloads.trace_random(rng, n, nv, p=[0.3, 0.35, 0.1, 0.1, 0.15])
                reqs.append((0, ks, var))
        sessions.append((s, nv, reqs))
    return sessions


def has_struct(tok):
    return bool(np.isin(tok & 15, [8, 10]).any())


def oracle_results(oracle_mod, sessions):
    """Each session run in order on the oracle from all-{(V,I)} sets: a trace
    while every set is a singleton is a trace check on status codes (results
    are codes); a program, or a trace after a program with If / While, is a
    relation-mode check (results are masks).  Returns the per-request results
    and each session's final masks."""
    out, finals = {}, {}
    for sid, nv, reqs in sessions:
        masks = np.full(nv, 1 << 1, np.uint8)
        det = True
        for i, (kind, a, b) in enumerate(reqs):
            if kind == 0 and det:
                codes = (np.log2(masks).astype(np.uint8))
                step, st, vff, ff = oracle_mod.check_trace(a, b, nv, init_status=codes)
                masks = (1 << st.astype(np.int64)).astype(np.uint8)
                out[(sid, i)] = (step, ff, False)
            else:
                step, masks, ff = oracle_mod.check_program(a, b, nv, init_mask=masks)
                out[(sid, i)] = (step, ff, True)
                if kind == 1 and has_struct(a):
                    det = False
        finals[sid] = masks
    return out, finals


def run_server(amc, sessions, slots, one_at_a_time):
    res = {}
    with amc.Server(mem_budget_bytes=1 << 30, max_slots=slots) as srv:
        pending = {}
        order = [(sid, nv, i, r) for sid, nv, reqs in sessions for i, r in enumerate(reqs)]
        if not one_at_a_time:      # interleave sessions: round robin by request index
            order.sort(key=lambda x: (x[2], x[0]))
        for sid, nv, i, (kind, a, b) in order:
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
        finals = {sid: srv.export(sid, nv) for sid, nv, _ in sessions}
    return res, finals


def test_alone_equals_mix_equals_oracle(amc, oracle_mod):
    sessions = make_sessions()
    exp, exp_fin = oracle_results(oracle_mod, sessions)
    assert any(m for (_, _, m) in exp.values()) and any(not m for (_, _, m) in exp.values())
    alone, fin_a = run_server(amc, sessions, slots=1, one_at_a_time=True)
    mix, fin_m = run_server(amc, sessions, slots=16, one_at_a_time=False)
    for key, (step, ff, is_mask) in exp.items():
        for got in (alone[key], mix[key]):
            assert got["error"] == 0
            assert got["is_mask"] == is_mask, key
            assert np.array_equal(got["status"], step), key
            assert got["first_fault"] == ff, key
    for sid in exp_fin:
        assert np.array_equal(fin_a[sid], exp_fin[sid]), sid
        assert np.array_equal(fin_m[sid], exp_fin[sid]), sid


def test_rejects_malformed_requests(amc):
    with amc.Server(mem_budget_bytes=1 << 26, max_slots=2) as srv:
        t = srv.submit(1, 0, 4, np.array([0, 1], np.uint8), np.array([0, 9], np.int32))   # checked on the device
        while (r := srv.poll(t)) is None:
            time.sleep(1e-4)
        assert r["error"] == amc.E_RANGE
        t = srv.submit(4, 0, 4, np.array([0, 0x21], np.uint8), np.array([0, 1], np.int32))
        while (r := srv.poll(t)) is None:
            time.sleep(1e-4)
        assert r["error"] == amc.E_INVALID
        with pytest.raises(amc.AmcError):
            srv.submit(2, 1, 4, np.array([8, 0], np.uint8), np.array([1, 0], np.int32))
        t = srv.submit(3, 0, 4, np.array([1, 4], np.uint8), np.array([0, 0], np.int32))
        while (r := srv.poll(t)) is None:
            time.sleep(1e-4)
        assert r["status"].tolist() == [1, 1] and r["first_fault"] == -1 and not r["is_mask"]
        with pytest.raises(amc.AmcError):           # a session keeps its variable count
            srv.submit(3, 1, 5, np.array([0], np.uint8), np.array([0], np.int32))
        t = srv.submit(3, 1, 4, np.array([0], np.uint8), np.array([0], np.int32))   # a program after a trace
        while (r := srv.poll(t)) is None:
            time.sleep(1e-4)
        assert r["status"].tolist() == [1 << 1] and r["is_mask"]
        assert srv.export(3, 4).tolist() == [1 << 1] * 4


def test_borrowed_buffers(amc, oracle_mod):
    # AMC_REQ_BORROW: pinned tensors read when the request runs (no copy at
    # submission); results as for copied requests and as the oracle's
    import torch
    rng = np.random.default_rng(8)
    ks, var = workloads.trace_random(rng, 200_000, 500)
    kt, vt = torch.from_numpy(ks).pin_memory(), torch.from_numpy(var).pin_memory()
    with amc.Server(mem_budget_bytes=1 << 30, max_slots=4) as srv:
        t1 = srv.submit(1, 0, 500, kt, vt, borrow=True)
        t2 = srv.submit(2, 0, 500, ks, var)
        res = {}
        while len(res) < 2:
            for t in (t1, t2):
                if t not in res and (r := srv.poll(t)) is not None:
                    res[t] = r
            time.sleep(1e-4)
    step, final, vff, ff = oracle_mod.check_trace(ks, var, 500)
    for t in (t1, t2):
        assert res[t]["error"] == 0 and np.array_equal(res[t]["status"], step) and res[t]["first_fault"] == ff


def test_completed_reports_each_ticket_once(amc, oracle_mod):
    # amc_serve_completed: every finished ticket exactly once, results as the
    # oracle's, many sessions in flight at once
    rng = np.random.default_rng(9)
    reqs = []
    with amc.Server(mem_budget_bytes=1 << 30, max_slots=8) as srv:
        for i in range(60):
            n = int(rng.integers(1, 50_000))
            ks, var = workloads.trace_random(rng, n, 300)
            while (t := srv.submit(100 + i % 13, 0, 300, ks, var)) is None:
                time.sleep(1e-4)
            reqs.append((t, i % 13, ks, var))
        seen, res = [], {}
        deadline = time.time() + 60
        while len(seen) < len(reqs) and time.time() < deadline:
            for t in srv.completed(cap=7):
                seen.append(t)
                res[t] = srv.poll(t)
            time.sleep(1e-4)
        assert sorted(seen) == sorted(t for t, *_ in reqs)
        assert srv.completed() == []
    # per session, requests chain from the previous statuses
    for sess in range(13):
        mine = [r for r in reqs if r[1] == sess]
        ks = np.concatenate([r[2] for r in mine])
        var = np.concatenate([r[3] for r in mine])
        step, *_ = oracle_mod.check_trace(ks, var, 300)
        got = np.concatenate([res[r[0]]["status"] for r in mine])
        assert np.array_equal(got, step)
