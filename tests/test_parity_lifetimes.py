"""GPU parity of the VectorPU path over pvectors with lifetimes
(amc_vectorpu_overlap_pairs, amc_translate_vectorpu_lifetimes,
amc_check_inherited_trace) with the oracle (oracle_vectorpu_lifetimes): the
translated trace (op bytes, ids, call offsets, creation records) and every
status, final status and first fault bit-exact.  Covers the seeded lifetimes
workload at reduced sizes (several vectors, thousands of pvectors, calls
across many tiles), the Section 4.3 example with deletions, the reduction to
the static path, malformed lifetimes and links, dead operands, an
over-small pair capacity, and the full-size workload through properties that
hold at any size."""
import numpy as np
import pytest
import torch

import workloads

pytestmark = pytest.mark.gpu
R, W, RW = 1, 2, 3
K_NOOP = 4
II, VI, IV, VV, F = 0, 1, 2, 3, 4


@pytest.fixture(scope="module")
def amc():
    import paper_1910_11110_gb300 as m
    m.build()
    return m


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def gpu_run(amc, w, infer=True, max_pairs=None):
    d = {k: dev(v) for k, v in w.items()}
    tr = amc.translate_vectorpu_lifetimes(d["arr_start"], d["arr_len"], d["arr_parent"], d["arr_born"],
                                          d["arr_died"], d["call_side"], d["call_off"], d["opnd_array"],
                                          d["opnd_mode"], infer_overlap=infer, max_pairs=max_pairs)
    A = w["arr_start"].size
    ck = amc.check_inherited_trace(tr["kind_side"], tr["var"], A, d["arr_parent"], tr["arr_probe"])
    code = amc.sync_status()
    return tr, ck, code


def compare(amc, oracle_mod, w, infer=True):
    exp = oracle_mod.vectorpu_lifetimes(**w, infer_overlap=infer)
    tr, ck, code = gpu_run(amc, w, infer)
    assert code == 0
    assert tr["n"] == exp["kind_side"].size
    assert np.array_equal(tr["kind_side"].cpu().numpy(), exp["kind_side"])
    assert np.array_equal(tr["var"].cpu().numpy(), exp["var"])
    assert np.array_equal(tr["call_first_op"].cpu().numpy(), exp["call_first_op"])
    assert np.array_equal(tr["arr_probe"].cpu().numpy(), exp["arr_probe"])
    step = ck["step_status"].cpu().numpy()
    bad = np.nonzero(step != exp["step_status"])[0]
    assert bad.size == 0, bad[:10]
    assert np.array_equal(ck["final_status"].cpu().numpy(), exp["final_status"])
    assert np.array_equal(ck["var_first_fault"].cpu().numpy(), exp["var_first_fault"])
    assert int(ck["first_fault"].cpu()[0]) == exp["first_fault"]
    return exp


@pytest.mark.parametrize("kw", [
    dict(seed=61, n_vectors=4, vec_len=1 << 12, n_pvectors=600, n_calls=3000),
    dict(seed=62, n_vectors=16, vec_len=1 << 14, n_pvectors=4096, n_calls=1 << 15, len_log2=(4.0, 12.0)),
    dict(seed=63, n_vectors=1, vec_len=1 << 16, n_pvectors=2000, n_calls=1 << 14, mean_life=200.0),
    dict(seed=64, n_vectors=8, vec_len=1 << 16, n_pvectors=8192, n_calls=1 << 17, drop_p=0.01),
    dict(seed=65, n_vectors=3, vec_len=1 << 10, n_pvectors=300, n_calls=4000, max_opnds=12),
])
def test_lifetimes_workloads(amc, oracle_mod, kw):
    w = workloads.vectorpu_lifetimes(**kw)
    exp = compare(amc, oracle_mod, w)
    assert (exp["arr_probe"] >= 0).sum() >= kw["n_pvectors"] // 2


def test_without_inference(amc, oracle_mod):
    w = workloads.vectorpu_lifetimes(seed=66, n_vectors=4, vec_len=1 << 12, n_pvectors=800, n_calls=5000)
    compare(amc, oracle_mod, w, infer=False)


def test_live_throughout_equals_static_path(amc, oracle_mod):
    # every array live for the whole run, no pvector: the static translation
    w0 = workloads.vectorpu_calls(seed=67, n_arrays=300, space=1 << 14, n_calls=20_000, len_log2=(2.0, 10.0))
    A, C = w0["arr_start"].size, w0["call_side"].size
    w = dict(w0, arr_parent=np.full(A, -1, np.int32), arr_born=np.zeros(A, np.int32),
             arr_died=np.full(A, C, np.int32))
    compare(amc, oracle_mod, w)
    d = {k: dev(v) for k, v in w0.items()}
    st = amc.translate_vectorpu(d["arr_start"], d["arr_len"], d["call_side"], d["call_off"], d["opnd_array"],
                                d["opnd_mode"])
    tr, _, code = gpu_run(amc, w)
    assert code == 0
    assert torch.equal(st["kind_side"], tr["kind_side"]) and torch.equal(st["var"], tr["var"])


def test_section4_3_example_with_deletion(amc, oracle_mod):
    # v = [0, 10) and pv1 = [2:5], pv2 = [4:8], pv3 = [7:9], pv4 = [2:3] its
    # pvectors; pv2 deleted after f1, pv3 created before f2
    w = dict(arr_start=np.array([2, 4, 7, 2, 0], np.int32), arr_len=np.array([3, 4, 2, 1, 10], np.int32),
             arr_parent=np.array([4, 4, 4, 4, -1], np.int32), arr_born=np.array([0, 0, 1, 0, 0], np.int32),
             arr_died=np.array([3, 1, 3, 3, 3], np.int32), call_side=np.array([0, 1, 0], np.uint8),
             call_off=np.array([0, 2, 3, 4], np.int32), opnd_array=np.array([0, 1, 2, 3], np.int32),
             opnd_mode=np.array([R, R, W, RW], np.uint8))
    exp = compare(amc, oracle_mod, w)
    assert list(exp["arr_probe"]) == [0, 2, exp["call_first_op"][1], 4, -1]


@pytest.mark.parametrize("case,code", [
    ("dead_operand", "E_INVALID"), ("late_parent", "E_INVALID"), ("parent_range", "E_RANGE"),
    ("outside_parent", "E_INVALID"), ("pvector_parent", "E_INVALID"), ("empty_life", "E_INVALID"),
])
def test_malformed_reported(amc, case, code):
    w = dict(arr_start=np.array([0, 2], np.int32), arr_len=np.array([10, 3], np.int32),
             arr_parent=np.array([-1, 0], np.int32), arr_born=np.array([0, 1], np.int32),
             arr_died=np.array([2, 2], np.int32), call_side=np.array([0, 0], np.uint8),
             call_off=np.array([0, 1, 2], np.int32), opnd_array=np.array([0, 1], np.int32),
             opnd_mode=np.array([R, R], np.uint8))
    if case == "dead_operand":
        w["opnd_array"] = np.array([1, 0], np.int32)           # pvector 1 used at call 0, born at 1
    elif case == "late_parent":
        w["arr_born"] = np.array([1, 0], np.int32)
        w["opnd_array"] = np.array([1, 0], np.int32)
    elif case == "parent_range":
        w["arr_parent"] = np.array([-1, 7], np.int32)
    elif case == "outside_parent":
        w["arr_start"] = np.array([0, 9], np.int32)
    elif case == "pvector_parent":
        w["arr_parent"] = np.array([1, 0], np.int32)
    elif case == "empty_life":
        w["arr_born"] = np.array([0, 2], np.int32)
    assert amc.sync_status() == 0
    # the first error latched is the translation's (the check may add its own)
    _, _, got = gpu_run(amc, w, max_pairs=16)
    assert got == getattr(amc, code)
    assert amc.sync_status() == 0


def test_pair_capacity_exceeded(amc):
    w = workloads.vectorpu_lifetimes(seed=68, n_vectors=2, vec_len=1 << 10, n_pvectors=200, n_calls=1000)
    d = {k: dev(v) for k, v in w.items()}
    C = w["call_side"].size
    need = int(amc.vectorpu_overlap_pairs(d["arr_start"], d["arr_len"], d["arr_born"], d["arr_died"], C).item())
    assert need > 10
    amc.sync_status()
    amc.translate_vectorpu_lifetimes(d["arr_start"], d["arr_len"], d["arr_parent"], d["arr_born"], d["arr_died"],
                                     d["call_side"], d["call_off"], d["opnd_array"], d["opnd_mode"],
                                     max_pairs=need - 1)
    assert amc.sync_status() == amc.E_RANGE
    # every pair, once, when the lifetimes are left out (count only)
    allp = int(amc.vectorpu_overlap_pairs(d["arr_start"], d["arr_len"]).item())
    assert allp > 0
    assert amc.sync_status() == 0


def test_overlap_pair_count_matches_brute_force(amc):
    rng = np.random.default_rng(69)
    A = 500
    s = rng.integers(0, 2000, A).astype(np.int32)
    ln = rng.integers(1, 120, A).astype(np.int32)
    b = rng.integers(0, 90, A).astype(np.int32)
    e = (b + rng.integers(1, 30, A)).astype(np.int32)
    ov = (s[:, None] < (s + ln)[None, :]) & (s[None, :] < (s + ln)[:, None])
    meet = np.maximum(b[:, None], b[None, :]) < np.minimum(e[:, None], e[None, :])
    np.fill_diagonal(ov, False)
    # one entry per time bucket the two lifetimes share: 120 calls in 120
    # buckets of one call; 1,000 calls in 256 buckets of 4 calls
    lo, hi = np.maximum(b[:, None], b[None, :]), np.minimum(e[:, None], e[None, :])
    for C, bl in ((120, 1), (1000, 4)):
        nb = np.where(ov & meet, (hi - 1) // bl - lo // bl + 1, 0)
        got = amc.vectorpu_overlap_pairs(dev(s), dev(ln), dev(b), dev(e), C).item()
        assert got == int(nb.sum())
    assert amc.vectorpu_overlap_pairs(dev(s), dev(ln)).item() == int(ov.sum())
    assert amc.sync_status() == 0


def test_full_size_workload_properties(amc):
    """The seeded workload at full size (2^24 calls, 16 vectors of 2^20
    elements, 65,536 pvectors): no error; one creation record per pvector,
    each Noop v, Noop v# on its vector at the head of its creation call; the
    abstract variables never (I,I) nor stuck (Property Safety carried to
    them); first fault = the smallest per-variable first fault, which is an
    op on that variable that is stuck."""
    w = workloads.vectorpu_lifetimes()
    A = w["arr_start"].size
    tr, ck, code = gpu_run(amc, w)
    assert code == 0
    probe = tr["arr_probe"].cpu().numpy()
    par = w["arr_parent"]
    kids = par >= 0
    assert (probe[~kids] == -1).all() and (probe[kids] >= 0).all()
    pr = torch.from_numpy(probe[kids]).cuda()
    v = tr["var"]
    assert torch.equal(v[pr].cpu(), torch.from_numpy(par[kids]))
    assert torch.equal(v[pr + 1].cpu(), torch.from_numpy(par[kids] + A))
    assert bool(((tr["kind_side"][pr] == K_NOOP) & (tr["kind_side"][pr + 1] == K_NOOP)).all())
    cfo = tr["call_first_op"].cpu().numpy()
    assert np.array_equal(np.searchsorted(cfo, probe[kids], side="right") - 1, w["arr_born"][kids])
    st = ck["step_status"]
    absm = v >= A
    assert not bool(((st == II) | (st == F))[absm].any())
    vff = ck["var_first_fault"].cpu().numpy()
    ff = int(ck["first_fault"].cpu()[0])
    has = vff >= 0
    assert ff == (int(vff[has].min()) if has.any() else -1)
    if ff >= 0:
        assert int(st[ff]) == F
        assert int(v[ff]) == int(np.argmin(np.where(has, vff, np.iinfo(np.int32).max)))
