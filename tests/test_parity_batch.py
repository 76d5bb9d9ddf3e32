"""GPU parity of amc_check_batch (relation mode: If = union, While = closure)
with the oracle: every step mask, final mask and program first fault is
bit-exact.  Covers nesting up to the depth limit, empty branches and bodies,
programs with more variables than the shared-memory table holds, graph replay,
malformed programs, and the 100,000-program workload."""
import numpy as np
import pytest
import torch

import workloads

pytestmark = pytest.mark.gpu
IF, ELSE, WHILE, END = 8, 9, 10, 11


@pytest.fixture(scope="module")
def amc():
    import paper_1910_11110_gb300 as m
    m.build()
    return m


def run(amc, b, graph=False):
    dev = torch.device("cuda")
    t = lambda a: torch.from_numpy(np.ascontiguousarray(a)).to(dev)
    out = amc.check_batch(t(b["tok"]), t(b["payload"]), t(b["prog_tok_off"]), t(b["prog_nvars"]),
                          graph_capture=graph, stream=torch.cuda.current_stream() if graph else None)
    assert amc.sync_status() == 0
    return {k: v.cpu().numpy() for k, v in out.items()}


def compare(amc, oracle_mod, b, graph=False):
    step, final, pff = oracle_mod.check_batch(b["tok"], b["payload"], b["prog_tok_off"], b["prog_nvars"])
    got = run(amc, b, graph)
    assert np.array_equal(got["step_mask"], step), np.nonzero(got["step_mask"] != step)[0][:10]
    assert np.array_equal(got["final_mask"], final)
    assert np.array_equal(got["prog_first_fault"], pff)


@pytest.mark.parametrize("kw", [
    dict(n_progs=200, seed=41, median=300.0, max_len=5000, vars_lo=2, vars_hi=40),
    dict(n_progs=300, seed=42, median=200.0, max_len=3000, vars_lo=1, vars_hi=3, p_if=0.2, p_while=0.15),
    dict(n_progs=50, seed=43, median=2000.0, max_len=20000, vars_lo=64, vars_hi=4096),
    dict(n_progs=20, seed=44, median=500.0, max_len=4000, vars_lo=5000, vars_hi=9000),
    dict(n_progs=100, seed=45, median=100.0, max_len=2000, vars_lo=3, vars_hi=8, p_if=0.3, p_while=0.3,
         max_depth=8, max_branch=6, max_body=6),
])
def test_random_batches(amc, oracle_mod, kw):
    compare(amc, oracle_mod, workloads.programs(**kw))


def test_graph_replay_matches(amc, oracle_mod):
    b = workloads.programs(n_progs=400, seed=46, median=500.0, max_len=8000)
    compare(amc, oracle_mod, b, graph=True)
    compare(amc, oracle_mod, b, graph=True)      # second call replays the cached graph


def test_edge_programs(amc, oracle_mod):
    progs = [
        ([], []),                                                   # empty program
        ([IF, ELSE, END], [0, 0, 0]),                                # empty branches
        ([WHILE, END, 1 | 16], [0, 0, 0]),                           # empty body
        ([WHILE, 1 | 16, 2, END], [2, 0, 0, 0]),                     # closure reaches a fault
        ([IF, 1, ELSE, 1 | 16, END, 0, 0 | 16], [1, 0, 1, 0, 0, 0, 0]),
    ]
    tok = np.array([x for p, _ in progs for x in p], np.uint8)
    pay = np.array([x for _, q in progs for x in q], np.int32)
    off = np.concatenate([[0], np.cumsum([len(p) for p, _ in progs])]).astype(np.int64)
    b = dict(tok=tok, payload=pay, prog_tok_off=off, prog_nvars=np.array([1, 1, 1, 1, 1], np.int32))
    compare(amc, oracle_mod, b)


def test_malformed_reported(amc):
    dev = torch.device("cuda")
    t = lambda a, dt: torch.tensor(a, dtype=dt, device=dev)
    amc.check_batch(t([IF, 0], torch.uint8), t([1, 0], torch.int32), t([0, 2], torch.int64), t([1], torch.int32))
    assert amc.sync_status() == amc.E_INVALID
    amc.check_batch(t([0], torch.uint8), t([3], torch.int32), t([0, 1], torch.int64), t([1], torch.int32))
    assert amc.sync_status() == amc.E_RANGE
    assert amc.sync_status() == 0


def test_programs_workload_full_size(amc, oracle_mod):
    """100,000 programs, 64-4,096 vars, lognormal lengths (seed 3)."""
    compare(amc, oracle_mod, workloads.programs())


def _concat(progs):
    tok = np.concatenate([p[0] for p in progs]).astype(np.uint8)
    pay = np.concatenate([p[1] for p in progs]).astype(np.int32)
    off = np.concatenate([[0], np.cumsum([len(p[0]) for p in progs])]).astype(np.int64)
    nv = np.array([p[2] for p in progs], np.int32)
    return dict(tok=tok, payload=pay, prog_tok_off=off, prog_nvars=nv)


@pytest.fixture
def split8k(monkeypatch):
    # segments of 8,192 tokens (the default splits only far longer programs)
    monkeypatch.setenv("AMC_BATCH_SPLIT", "8192")


def test_split_programs(amc, oracle_mod, split8k):
    # programs longer than one segment (8,192 tokens) are cut at top-level
    # boundaries and checked as segments (relations of the earlier segments,
    # carried entry sets); lengths 8,193 .. 60,000 tokens, dense constructs so
    # that cuts land next to Ifs and Whiles, few and many variables, plus short
    # programs in between
    progs = []
    for i, (n, nv, pif, pwh) in enumerate([(9000, 4, 0.1, 0.1), (20000, 64, 0.05, 0.03), (60000, 4096, 0.02, 0.02),
                                           (8193, 1, 0.3, 0.2), (33000, 300, 0.2, 0.15)]):
        b = workloads.programs(1, seed=700 + i, median=float(n), sigma=0.001, max_len=n, vars_lo=nv, vars_hi=nv,
                               p_if=pif, p_while=pwh)
        progs.append((b["tok"], b["payload"], nv))
        s = workloads.programs(3, seed=800 + i, median=50.0, vars_lo=5, vars_hi=9)
        for k in range(3):
            a, z = s["prog_tok_off"][k], s["prog_tok_off"][k + 1]
            progs.append((s["tok"][a:z], s["payload"][a:z], int(s["prog_nvars"][k])))
    b = _concat(progs)
    assert b["prog_tok_off"][3] - b["prog_tok_off"][2] >= 0
    compare(amc, oracle_mod, b)
    compare(amc, oracle_mod, b, graph=True)


def test_split_program_without_boundaries(amc, oracle_mod, split8k):
    # one While around 20,000 tokens: no top-level boundary after the first
    # token, so every slot but the first stays empty and the program runs as one
    # segment; then the same body after 9,000 top-level ops (one cut)
    inner = workloads.programs(1, seed=710, median=20000.0, sigma=0.001, max_len=20000, vars_lo=50, vars_hi=50)
    body_t, body_p = inner["tok"], inner["payload"]
    whole_t = np.concatenate([[WHILE], body_t, [END]])
    whole_p = np.concatenate([[len(body_t)], body_p, [0]])
    ops = workloads.programs(1, seed=711, median=9000.0, sigma=0.001, max_len=9000, vars_lo=50, vars_hi=50, p_if=0.0,
                             p_while=0.0)
    second_t = np.concatenate([ops["tok"], whole_t])
    second_p = np.concatenate([ops["payload"], whole_p])
    compare(amc, oracle_mod, _concat([(whole_t, whole_p, 50), (second_t, second_p, 50)]))


def test_initial_masks_with_split_programs(amc, oracle_mod, split8k):
    # through the server, whose program requests start from the session's
    # sets: a short structured program leaves sets of several statuses, then a
    # 30,000-token program (split into segments) starts from them
    import time
    first = workloads.programs(1, seed=712, median=400.0, vars_lo=100, vars_hi=100, p_if=0.3, p_while=0.2)
    b = workloads.programs(1, seed=713, median=30000.0, sigma=0.001, max_len=30000, vars_lo=100, vars_hi=100)
    s1, m1, f1 = oracle_mod.check_program(first["tok"], first["payload"], 100)
    s2, m2, f2 = oracle_mod.check_program(b["tok"], b["payload"], 100, init_mask=m1)
    assert (np.bitwise_count(m1) > 1).any()
    with amc.Server(mem_budget_bytes=1 << 30, max_slots=2) as srv:
        res = []
        for prog in (first, b):
            t = srv.submit(9, 1, 100, prog["tok"], prog["payload"])
            while (r := srv.poll(t)) is None:
                time.sleep(1e-4)
            res.append(r)
        fin = srv.export(9, 100)
    assert res[0]["error"] == 0 and np.array_equal(res[0]["status"], s1) and res[0]["first_fault"] == f1
    assert res[1]["error"] == 0 and np.array_equal(res[1]["status"], s2) and res[1]["first_fault"] == f2
    assert np.array_equal(fin, m2)
