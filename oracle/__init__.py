"""CPU oracle of the access-mode consistency calculus (arXiv 1910.11110).

TEST INFRASTRUCTURE ONLY.  This package is imported by ``tests/``, by
``__graft_entry__.smoke()`` and by the ``cpu_baseline`` / ``--impl reference``
legs of ``bench.py``; the product library never imports it.  It wraps the
plain C interpreter in ``oracle.c`` (one op at a time, effects applied by
unification with the Section 3.1 signatures) with numpy-array helpers.
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "liboracle.so")
_lib = None

F = 4  # stuck status code


def build(force: bool = False) -> str:
    """Compile oracle.c into oracle/_build/liboracle.so (gcc, portable flags)."""
    src = os.path.join(_HERE, "oracle.c")
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(src)
            and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(os.path.join(_HERE, "oracle.h"))):
        return _LIB_PATH
    os.makedirs(_BUILD, exist_ok=True)
    tmp = _LIB_PATH + f".tmp{os.getpid()}"
    subprocess.check_call(["gcc", "-O2", "-std=c11", "-Wall", "-shared", "-fPIC",
                           "-o", tmp, src])
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def lib():
    global _lib
    if _lib is None:
        _lib = ctypes.CDLL(build())
        P = ctypes.c_void_p
        i64, i32 = ctypes.c_int64, ctypes.c_int32
        _lib.oracle_apply.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int]
        _lib.oracle_check_trace.argtypes = [P, P, i64, i32, P, P, P, P, P]
        _lib.oracle_check_trace_shard.argtypes = [P, P, i64, i32, i32, i32, P, P, P, P]
        _lib.oracle_check_program.argtypes = [P, P, i64, i32, P, P, P, P]
        _lib.oracle_check_batch.argtypes = [P, P, P, P, P, i64, P, P, P]
        _lib.oracle_overlaps.argtypes = [P, P, i32, P, P, i64]
        _lib.oracle_vectorpu.argtypes = [P, P, i32, P, P, i64, P, P, ctypes.c_int,
                                         P, P, i64, P, P, P, P, P, P]
        _lib.oracle_check_program_guarded.argtypes = [P, P, i64, i32, i32, P, P, P, P]
        _lib.oracle_check_batch_guarded.argtypes = [P, P, P, P, P, P, i64, P, P, P]
        _lib.oracle_vectorpu_lifetimes.argtypes = [P, P, P, P, P, i32, P, P, i64, P, P, ctypes.c_int,
                                                   P, P, i64, P, P, P, P, P, P, P]
        _lib.oracle_well_declared.argtypes = [P, i32, P, P, i64, P, P, P, P, P, P, P, P]
        _lib.oracle_apply_k.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int]
        _lib.oracle_check_trace_k.argtypes = [P, P, i64, i32, i32, P, P, P, P, P]
    return _lib


class OracleError(RuntimeError):
    pass


def _ptr(a):
    return None if a is None else a.ctypes.data_as(ctypes.c_void_p)


def _check(rc):
    if rc != 0:
        raise OracleError(f"oracle rejected the input (code {rc})")


def apply(kind: int, side: int, status: int) -> int:
    return lib().oracle_apply(kind, side, status)


def check_trace(kind_side, var, n_vars, init_status=None):
    """Trace mode.  Returns (step_status, final_status, var_first_fault, first_fault)."""
    ks = np.ascontiguousarray(kind_side, dtype=np.uint8)
    v = np.ascontiguousarray(var, dtype=np.int32)
    n = ks.shape[0]
    init = None if init_status is None else np.ascontiguousarray(init_status, dtype=np.uint8)
    step = np.empty(n, np.uint8)
    final = np.empty(n_vars, np.uint8)
    vff = np.empty(n_vars, np.int32)
    ff = np.empty(1, np.int64)
    _check(lib().oracle_check_trace(_ptr(ks), _ptr(v), n, n_vars, _ptr(init),
                                    _ptr(step), _ptr(final), _ptr(vff), _ptr(ff)))
    return step, final, vff, int(ff[0])


def check_trace_sharded(kind_side, var, n_vars, n_threads):
    """Trace mode on n_threads host threads: thread t runs the oracle over the
    whole trace for the variables v % n_threads == t (the ctypes calls release
    the GIL).  Same outputs as check_trace with all-(V,I) initial statuses."""
    import threading
    ks = np.ascontiguousarray(kind_side, dtype=np.uint8)
    v = np.ascontiguousarray(var, dtype=np.int32)
    n = ks.shape[0]
    step = np.empty(n, np.uint8)
    final = np.empty(n_vars, np.uint8)
    vff = np.empty(n_vars, np.int32)
    ffs = np.empty(n_threads, np.int64)
    rcs = [0] * n_threads
    L = lib()

    def run(t):
        rcs[t] = L.oracle_check_trace_shard(_ptr(ks), _ptr(v), n, n_vars, n_threads, t, _ptr(step), _ptr(final),
                                            _ptr(vff), ffs[t:].ctypes.data_as(ctypes.c_void_p))

    th = [threading.Thread(target=run, args=(t,)) for t in range(n_threads)]
    for x in th:
        x.start()
    for x in th:
        x.join()
    for rc in rcs:
        _check(rc)
    f = ffs[ffs >= 0]
    return step, final, vff, int(f.min()) if f.size else -1


KL_F = 0x80  # stuck status of the k-location check


def apply_k(op: int, status: int, k: int) -> int:
    return lib().oracle_apply_k(op, status, k)


def check_trace_k(op, var, n_vars, k, init_status=None):
    """Traces over k memory locations.  Returns (step_status, final_status,
    var_first_fault, first_fault); statuses are bit masks of valid locations,
    0x80 = stuck."""
    o = np.ascontiguousarray(op, dtype=np.uint8)
    v = np.ascontiguousarray(var, dtype=np.int32)
    n = o.shape[0]
    init = None if init_status is None else np.ascontiguousarray(init_status, dtype=np.uint8)
    step = np.empty(n, np.uint8)
    final = np.empty(n_vars, np.uint8)
    vff = np.empty(n_vars, np.int32)
    ff = np.empty(1, np.int64)
    _check(lib().oracle_check_trace_k(_ptr(o), _ptr(v), n, n_vars, k, _ptr(init), _ptr(step), _ptr(final),
                                      _ptr(vff), _ptr(ff)))
    return step, final, vff, int(ff[0])


def check_program(tok, payload, n_vars, init_mask=None):
    """Relation mode for one program.  Returns (step_mask, final_mask, first_fault)."""
    t = np.ascontiguousarray(tok, dtype=np.uint8)
    p = np.ascontiguousarray(payload, dtype=np.int32)
    init = None if init_mask is None else np.ascontiguousarray(init_mask, dtype=np.uint8)
    step = np.zeros(t.shape[0], np.uint8)
    final = np.empty(n_vars, np.uint8)
    ff = np.empty(1, np.int64)
    _check(lib().oracle_check_program(_ptr(t), _ptr(p), t.shape[0], n_vars, _ptr(init),
                                      _ptr(step), _ptr(final), _ptr(ff)))
    return step, final, int(ff[0])


def check_batch(tok, payload, prog_tok_off, prog_nvars):
    """Relation mode over a CSR batch.  Returns (step_mask, final_mask, prog_first_fault)."""
    t = np.ascontiguousarray(tok, dtype=np.uint8)
    p = np.ascontiguousarray(payload, dtype=np.int32)
    to = np.ascontiguousarray(prog_tok_off, dtype=np.int64)
    nv = np.ascontiguousarray(prog_nvars, dtype=np.int32)
    vo = np.zeros(nv.shape[0] + 1, np.int64)
    np.cumsum(nv, out=vo[1:])
    step = np.zeros(t.shape[0], np.uint8)
    final = np.empty(int(vo[-1]), np.uint8)
    pff = np.empty(nv.shape[0], np.int64)
    _check(lib().oracle_check_batch(_ptr(t), _ptr(p), _ptr(to), _ptr(nv), _ptr(vo),
                                    nv.shape[0], _ptr(step), _ptr(final), _ptr(pff)))
    return step, final, pff


def check_program_guarded(tok, payload, n_vars, guard, init_mask=None):
    """Path-sensitive relation mode for one program (conditions on the guard
    variable `guard`, -1 none).  Returns (step_mask, final_mask, first_fault)."""
    t = np.ascontiguousarray(tok, dtype=np.uint8)
    p = np.ascontiguousarray(payload, dtype=np.int32)
    init = None if init_mask is None else np.ascontiguousarray(init_mask, dtype=np.uint8)
    step = np.zeros(t.shape[0], np.uint8)
    final = np.empty(max(n_vars, 1), np.uint8)
    ff = np.empty(1, np.int64)
    _check(lib().oracle_check_program_guarded(_ptr(t), _ptr(p), t.shape[0], n_vars, int(guard), _ptr(init),
                                              _ptr(step), _ptr(final), _ptr(ff)))
    return step, final[:n_vars], int(ff[0])


def check_batch_guarded(tok, payload, prog_tok_off, prog_nvars, prog_guard):
    """Path-sensitive relation mode over a CSR batch.  Returns (step_mask,
    final_mask, prog_first_fault)."""
    t = np.ascontiguousarray(tok, dtype=np.uint8)
    p = np.ascontiguousarray(payload, dtype=np.int32)
    to = np.ascontiguousarray(prog_tok_off, dtype=np.int64)
    nv = np.ascontiguousarray(prog_nvars, dtype=np.int32)
    gd = np.ascontiguousarray(prog_guard, dtype=np.int32)
    vo = np.zeros(nv.shape[0] + 1, np.int64)
    np.cumsum(nv, out=vo[1:])
    step = np.zeros(t.shape[0], np.uint8)
    final = np.empty(max(int(vo[-1]), 1), np.uint8)
    pff = np.empty(nv.shape[0], np.int64)
    _check(lib().oracle_check_batch_guarded(_ptr(t), _ptr(p), _ptr(to), _ptr(nv), _ptr(vo), _ptr(gd), nv.shape[0],
                                            _ptr(step), _ptr(final), _ptr(pff)))
    return step, final[:int(vo[-1])], pff


def overlaps(arr_start, arr_len):
    """Overlap sets (CSR, ascending ids) of half-open intervals."""
    s = np.ascontiguousarray(arr_start, dtype=np.int32)
    ln = np.ascontiguousarray(arr_len, dtype=np.int32)
    n = s.shape[0]
    cap = max(1, n * n)
    off = np.empty(n + 1, np.int64)
    idx = np.empty(cap, np.int32)
    _check(lib().oracle_overlaps(_ptr(s), _ptr(ln), n, _ptr(off), _ptr(idx), cap))
    return off, idx[: off[-1]].copy()


def vectorpu(arr_start, arr_len, call_side, call_off, opnd_array, opnd_mode,
             infer_overlap=True, out_cap=None):
    """Translate and check VectorPU calls.

    Returns a dict with the translated trace (kind_side, var), call_first_op,
    step_status, final_status (2A), var_first_fault (2A) and first_fault.
    """
    s = np.ascontiguousarray(arr_start, dtype=np.int32)
    ln = np.ascontiguousarray(arr_len, dtype=np.int32)
    cs = np.ascontiguousarray(call_side, dtype=np.uint8)
    co = np.ascontiguousarray(call_off, dtype=np.int32)
    oa = np.ascontiguousarray(opnd_array, dtype=np.int32)
    om = np.ascontiguousarray(opnd_mode, dtype=np.uint8)
    A = s.shape[0]
    n_calls = cs.shape[0]
    if out_cap is None:
        out_cap = int(5 * oa.shape[0] + 48 * n_calls + 64)
    while True:
        ks = np.empty(out_cap, np.uint8)
        var = np.empty(out_cap, np.int32)
        step = np.empty(out_cap, np.uint8)
        n_out = np.empty(1, np.int64)
        cfo = np.empty(n_calls + 1, np.int64)
        final = np.empty(2 * A, np.uint8)
        vff = np.empty(2 * A, np.int32)
        ff = np.empty(1, np.int64)
        rc = lib().oracle_vectorpu(_ptr(s), _ptr(ln), A, _ptr(cs), _ptr(co), n_calls,
                                   _ptr(oa), _ptr(om), int(bool(infer_overlap)),
                                   _ptr(ks), _ptr(var), out_cap, _ptr(n_out), _ptr(cfo),
                                   _ptr(step), _ptr(final), _ptr(vff), _ptr(ff))
        if rc == -4 and out_cap < (1 << 40):
            out_cap *= 2
            continue
        _check(rc)
        n = int(n_out[0])
        return dict(kind_side=ks[:n].copy(), var=var[:n].copy(), step_status=step[:n].copy(),
                    call_first_op=cfo, final_status=final, var_first_fault=vff,
                    first_fault=int(ff[0]))


def vectorpu_lifetimes(arr_start, arr_len, arr_parent, arr_born, arr_died, call_side, call_off, opnd_array,
                       opnd_mode, infer_overlap=True, out_cap=None):
    """VectorPU calls over pvectors with lifetimes and inherited statuses.

    Returns the dict of vectorpu() plus arr_probe (int64 [A]: index of the
    Noop v, Noop v# pair recording each pvector's creation, -1 for vectors).
    """
    s = np.ascontiguousarray(arr_start, dtype=np.int32)
    ln = np.ascontiguousarray(arr_len, dtype=np.int32)
    par = np.ascontiguousarray(arr_parent, dtype=np.int32)
    bo = np.ascontiguousarray(arr_born, dtype=np.int32)
    di = np.ascontiguousarray(arr_died, dtype=np.int32)
    cs = np.ascontiguousarray(call_side, dtype=np.uint8)
    co = np.ascontiguousarray(call_off, dtype=np.int32)
    oa = np.ascontiguousarray(opnd_array, dtype=np.int32)
    om = np.ascontiguousarray(opnd_mode, dtype=np.uint8)
    A = s.shape[0]
    n_calls = cs.shape[0]
    if out_cap is None:
        out_cap = int(5 * oa.shape[0] + 48 * n_calls + 2 * A + 64)
    while True:
        ks = np.empty(out_cap, np.uint8)
        var = np.empty(out_cap, np.int32)
        step = np.empty(out_cap, np.uint8)
        n_out = np.empty(1, np.int64)
        cfo = np.empty(n_calls + 1, np.int64)
        probe = np.empty(A, np.int64)
        final = np.empty(2 * A, np.uint8)
        vff = np.empty(2 * A, np.int32)
        ff = np.empty(1, np.int64)
        rc = lib().oracle_vectorpu_lifetimes(_ptr(s), _ptr(ln), _ptr(par), _ptr(bo), _ptr(di), A, _ptr(cs),
                                             _ptr(co), n_calls, _ptr(oa), _ptr(om), int(bool(infer_overlap)),
                                             _ptr(ks), _ptr(var), out_cap, _ptr(n_out), _ptr(cfo), _ptr(probe),
                                             _ptr(step), _ptr(final), _ptr(vff), _ptr(ff))
        if rc == -4 and out_cap < (1 << 40):
            out_cap *= 2
            continue
        _check(rc)
        n = int(n_out[0])
        return dict(kind_side=ks[:n].copy(), var=var[:n].copy(), step_status=step[:n].copy(),
                    call_first_op=cfo, arr_probe=probe, final_status=final, var_first_fault=vff,
                    first_fault=int(ff[0]))


def well_declared(arr_loc_off, loc_owner, call_tok_off, tok, payload, call_am_off, am_array, am_mode):
    """Static well-declaredness of calls AM{S}.  Returns (violations uint32 [C],
    first_bad int64 [C], first_unmet int32 [C]); see oracle.h."""
    alo = np.ascontiguousarray(arr_loc_off, dtype=np.int64)
    own = np.ascontiguousarray(loc_owner, dtype=np.int32)
    cto = np.ascontiguousarray(call_tok_off, dtype=np.int64)
    t = np.ascontiguousarray(tok, dtype=np.uint8)
    p = np.ascontiguousarray(payload, dtype=np.int32)
    cao = np.ascontiguousarray(call_am_off, dtype=np.int64)
    aa = np.ascontiguousarray(am_array, dtype=np.int32)
    am = np.ascontiguousarray(am_mode, dtype=np.uint8)
    n_calls = cto.shape[0] - 1
    viol = np.empty(n_calls, np.uint32)
    bad = np.empty(n_calls, np.int64)
    unmet = np.empty(n_calls, np.int32)
    _check(lib().oracle_well_declared(_ptr(alo), alo.shape[0] - 1, _ptr(own), _ptr(cto), n_calls, _ptr(t), _ptr(p),
                                      _ptr(cao), _ptr(aa), _ptr(am), _ptr(viol), _ptr(bad), _ptr(unmet)))
    return viol, bad, unmet
