"""GPU parity of amc_translate_vectorpu + amc_check_guarded_trace with the
oracle's VectorPU mode: the translated statements (op bytes, variable ids,
call offsets) and every status are bit-exact."""
import numpy as np
import pytest
import torch

import workloads

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def amc():
    import paper_1910_11110_gb300 as m
    m.build()
    return m


def to_dev(w):
    dev = torch.device("cuda")
    return {k: torch.from_numpy(np.ascontiguousarray(v)).to(dev) for k, v in w.items()}


def run_gpu(amc, w, infer=True):
    d = to_dev(w)
    tr = amc.translate_vectorpu(d["arr_start"], d["arr_len"], d["call_side"], d["call_off"], d["opnd_array"],
                                d["opnd_mode"], infer_overlap=infer)
    assert amc.sync_status() == 0
    A = w["arr_start"].shape[0]
    out = amc.check_trace(tr["kind_side"], tr["var"], 2 * A, guarded=True)
    assert amc.sync_status() == 0
    return tr, out


def compare(amc, oracle_mod, w, infer=True):
    exp = oracle_mod.vectorpu(**w, infer_overlap=infer)
    tr, out = run_gpu(amc, w, infer)
    assert tr["n"] == len(exp["kind_side"])
    assert np.array_equal(tr["kind_side"].cpu().numpy(), exp["kind_side"])
    assert np.array_equal(tr["var"].cpu().numpy(), exp["var"])
    assert np.array_equal(tr["call_first_op"].cpu().numpy(), exp["call_first_op"])
    assert np.array_equal(out["step_status"].cpu().numpy(), exp["step_status"])
    assert np.array_equal(out["final_status"].cpu().numpy(), exp["final_status"])
    assert np.array_equal(out["var_first_fault"].cpu().numpy(), exp["var_first_fault"])
    assert int(out["first_fault"].cpu()[0]) == exp["first_fault"]


@pytest.mark.parametrize("seed,n_arrays,space,n_calls,drop", [
    (31, 8, 256, 500, 0.0), (32, 64, 1 << 14, 5000, 0.01), (33, 300, 1 << 18, 30_000, 1e-3),
    (34, 4096, 1 << 24, 40_000, 1e-4), (35, 1, 100, 50, 0.0), (36, 33, 1 << 10, 7000, 0.05)])
@pytest.mark.parametrize("infer", [True, False])
def test_random_calls(amc, oracle_mod, seed, n_arrays, space, n_calls, drop, infer):
    w = workloads.vectorpu_calls(seed=seed, n_arrays=n_arrays, space=space, n_calls=n_calls,
                                 len_log2=(2.0, 12.0), drop_p=drop)
    compare(amc, oracle_mod, w, infer)


def test_pvector_example(amc, oracle_mod):
    iv = [(2, 4), (4, 5), (7, 3), (2, 2)]
    w = dict(arr_start=np.array([a for a, _ in iv], np.int32), arr_len=np.array([b for _, b in iv], np.int32),
             call_side=np.array([0, 0, 0], np.uint8), call_off=np.array([0, 2, 3, 5], np.int32),
             opnd_array=np.array([0, 1, 2, 3, 1], np.int32), opnd_mode=np.array([1, 1, 2, 3, 1], np.uint8))
    compare(amc, oracle_mod, w)


def test_empty_calls(amc, oracle_mod):
    w = dict(arr_start=np.array([0, 5], np.int32), arr_len=np.array([10, 10], np.int32),
             call_side=np.zeros(0, np.uint8), call_off=np.zeros(1, np.int32),
             opnd_array=np.zeros(0, np.int32), opnd_mode=np.zeros(0, np.uint8))
    compare(amc, oracle_mod, w)


def test_malformed_calls_reported(amc):
    dev = torch.device("cuda")
    t = lambda a, dt: torch.tensor(a, dtype=dt, device=dev)
    amc.translate_vectorpu(t([0, 4], torch.int32), t([4, 4], torch.int32), t([0], torch.uint8),
                           t([0, 2], torch.int32), t([1, 1], torch.int32), t([1, 2], torch.uint8))
    assert amc.sync_status() == amc.E_INVALID       # duplicate operand
    amc.translate_vectorpu(t([0, 4], torch.int32), t([4, 4], torch.int32), t([0], torch.uint8),
                           t([0, 1], torch.int32), t([7], torch.int32), t([1], torch.uint8))
    assert amc.sync_status() == amc.E_RANGE         # array id out of range
    assert amc.sync_status() == 0


def test_vectorpu_workload_full_size(amc, oracle_mod):
    """4,096 intervals over 2^24, 2^24 calls, 1e-4 dropped annotations (seed 2):
    the whole translated trace and every status against the oracle."""
    w = workloads.vectorpu_calls(seed=2)
    compare(amc, oracle_mod, w)
