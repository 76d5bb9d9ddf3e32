"""GPU parity of the static well-declaredness check (amc_check_well_declared)
against the oracle: every violation bit, first bad token and first unmet
array, on the paper's examples, on generated calls with many injected flaws,
on arrays larger than one warp pass of tracked locations, on the default
2^20-call workload, and on malformed input (errors reported)."""
import json
import os

import numpy as np
import pytest
import torch

import workloads

pytestmark = pytest.mark.gpu
GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "section3_3_well_declared.json")


@pytest.fixture(scope="module")
def amc():
    import paper_1910_11110_gb300 as m
    m.build()
    return m


def gpu(amc, w):
    t = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()
    out = amc.check_well_declared(t(w["arr_loc_off"]), t(w["loc_owner"]), t(w["call_tok_off"]), t(w["tok"]),
                                  t(w["payload"]), t(w["call_am_off"]), t(w["am_array"]), t(w["am_mode"]))
    rc = amc.sync_status()
    return rc, out


def same(amc, oracle_mod, w):
    exp = oracle_mod.well_declared(**w)
    rc, out = gpu(amc, w)
    assert rc == 0
    got = (out["violations"].cpu().numpy().astype(np.uint32), out["first_bad"].cpu().numpy(),
           out["first_unmet"].cpu().numpy())
    for name, e, g in zip(("violations", "first_bad", "first_unmet"), exp, got):
        assert np.array_equal(e, g), (name, np.nonzero(e != g)[0][:10])
    return exp


def pack(arrays, calls):
    alo = np.zeros(len(arrays) + 1, np.int64)
    alo[1:] = np.cumsum(arrays)
    owner = np.repeat(np.arange(len(arrays)), arrays).astype(np.int32)
    cto, cao, tok, pay, aa, am = [0], [0], [], [], [], []
    for decl, body in calls:
        tok += [b for b, _ in body]
        pay += [p for _, p in body]
        aa += [a for a, _ in decl]
        am += [m for _, m in decl]
        cto.append(len(tok))
        cao.append(len(aa))
    return dict(arr_loc_off=alo, loc_owner=owner, call_tok_off=np.array(cto, np.int64),
                tok=np.array(tok, np.uint8), payload=np.array(pay, np.int32), call_am_off=np.array(cao, np.int64),
                am_array=np.array(aa, np.int32), am_mode=np.array(am, np.uint8))


def test_paper_examples(amc, oracle_mod):
    for case in json.load(open(GOLDEN))["cases"]:
        same(amc, oracle_mod, pack(case["arrays"], [(c["am"], c["body"]) for c in case["calls"]]))


@pytest.mark.parametrize("seed", [51, 52, 53])
def test_generated_calls_with_flaws(amc, oracle_mod, seed):
    w = workloads.wd_calls(n_calls=20_000, n_arrays=300, seed=seed, p_bad=0.4)
    exp = same(amc, oracle_mod, w)
    v = exp[0]
    assert all(((v >> k) & 1).sum() > 50 for k in range(4))


def test_arrays_past_one_warp_pass(amc, oracle_mod):
    # W arrays of up to 3,000 locations: the tracked bits take two or three
    # passes over the body
    w = workloads.wd_calls(n_calls=2_000, n_arrays=40, len_range=(1000, 3000), seed=54, p_bad=0.3)
    exp = same(amc, oracle_mod, w)
    assert (exp[0] & 8).any() and not (exp[0] == 0).all()


def test_default_workload(amc, oracle_mod):
    w = workloads.wd_calls()
    same(amc, oracle_mod, w)


def test_edge_cases(amc, oracle_mod):
    # empty bodies (a W declaration is then unmet), no declarations, nested
    # constructs at the deepest level, a While whose body writes (unmet)
    deep = []
    for _ in range(8):
        deep = [(10, 0)] + deep
    body_deep = [(8, 1), (1, 0), (9, 1), (1, 0), (11, 0)]
    for d in range(7):
        body_deep = [(8, len(body_deep)), *body_deep, (9, len(body_deep)), *body_deep, (11, 0)]
    calls = [([(0, 2)], []), ([], [(4, 0)]), ([], []), ([(0, 2)], body_deep),
             ([(0, 2)], [(10, 1), (1, 0), (11, 0)]), ([(1, 3)], [(0, 1), (1, 1)])]
    same(amc, oracle_mod, pack([1, 1], calls))
    same(amc, oracle_mod, pack([1], []))


def test_bad_input(amc):
    w = pack([2], [([(0, 3)], [(8, 1), (1, 0)])])             # If without ELSE / END
    assert gpu(amc, w)[0] == amc.E_INVALID
    w = pack([2], [([(0, 3)], [(1, 5)])])                     # location out of range
    assert gpu(amc, w)[0] == amc.E_RANGE
    w = pack([2], [([(0, 3)], [(6, 0)])])                     # GT in a body
    assert gpu(amc, w)[0] == amc.E_INVALID
    w = pack([1] * 40, [([(a, 1) for a in range(33)], [(0, 0)])])   # 33 declarations
    assert gpu(amc, w)[0] == amc.E_INVALID
    w = pack([2], [([(0, 7)], [(0, 0)])])                     # mode 7
    assert gpu(amc, w)[0] == amc.E_INVALID
    assert amc.sync_status() == 0
