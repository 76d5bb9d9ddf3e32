"""GB300 access-mode consistency checker: Python binding of the C ABI.

Thin ctypes layer over ``_build/libamc.so`` (see ``include/amc.h``): it only
marshals torch CUDA tensors into device pointers and sizes the workspaces; all
checking runs in the library's CUDA kernels.  There is no CPU fallback: the
functions raise ``RuntimeError`` when the library has not been built.
"""
from __future__ import annotations

import ctypes
import os

import torch

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_build", "libamc.so")
_lib = None

OK, E_INVALID, E_RANGE, E_NOMEM, E_TIMEOUT, E_CUDA, E_AGAIN = 0, -1, -2, -3, -4, -5, -6
ST_F = 4


class AmcError(RuntimeError):
    def __init__(self, code, what=""):
        self.code = code
        super().__init__(f"{what}: {error_string(code)} ({code})" if what else f"{error_string(code)} ({code})")


def build(force: bool = False) -> str:
    from . import builder
    return builder.build(force=force)


def lib():
    """The loaded CUDA library (raises if it is missing)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"CUDA library not built: {LIB_PATH} is missing "
                               "(run __graft_entry__.build() or paper_1910_11110_gb300.build())")
        L = ctypes.CDLL(LIB_PATH)
        P, i64, i32, sz, ci = ctypes.c_void_p, ctypes.c_int64, ctypes.c_int32, ctypes.c_size_t, ctypes.c_int
        L.amc_version.restype = ci
        L.amc_error_string.restype = ctypes.c_char_p
        L.amc_error_string.argtypes = [ci]
        L.amc_sync_status.argtypes = [P]
        L.amc_check_trace_workspace.restype = sz
        L.amc_check_trace_workspace.argtypes = [i64, i32]
        L.amc_check_trace.argtypes = [P, P, i64, i32, P, P, P, P, P, P, sz, P]
        L.amc_check_trace_plan.argtypes = [i64, i32, ci, P, P]
        L.amc_check_guarded_trace_workspace.restype = sz
        L.amc_check_guarded_trace_workspace.argtypes = [i64, i32]
        L.amc_check_guarded_trace.argtypes = [P, P, i64, i32, P, P, P, P, P, P, sz, P]
        L.amc_check_trace_host_workspace.restype = sz
        L.amc_check_trace_host_workspace.argtypes = [i64, i32, i64]
        L.amc_check_trace_host.argtypes = [P, P, i64, i32, P, P, P, P, P, i64, P, sz, P]
        if hasattr(L, "amc_translate_vectorpu"):
            L.amc_translate_vectorpu_workspace.restype = sz
            L.amc_translate_vectorpu_workspace.argtypes = [i32, i64, i64]
            L.amc_translate_vectorpu.argtypes = [P, P, i32, P, P, i64, P, P, i64, ci,
                                                 P, P, i64, P, P, P, sz, P]
        if hasattr(L, "amc_translate_vectorpu_lifetimes"):
            L.amc_vectorpu_overlap_pairs_workspace.restype = sz
            L.amc_vectorpu_overlap_pairs_workspace.argtypes = [i32, i64]
            L.amc_vectorpu_overlap_pairs.argtypes = [P, P, P, P, i32, i64, P, P, sz, P]
            L.amc_translate_vectorpu_lifetimes_workspace.restype = sz
            L.amc_translate_vectorpu_lifetimes_workspace.argtypes = [i32, i64, i64, i64]
            L.amc_translate_vectorpu_lifetimes.argtypes = [P, P, P, P, P, i32, P, P, i64, P, P, i64, ci, i64,
                                                           P, P, i64, P, P, P, P, sz, P]
            L.amc_check_inherited_trace_workspace.restype = sz
            L.amc_check_inherited_trace_workspace.argtypes = [i64, i32]
            L.amc_check_inherited_trace.argtypes = [P, P, i64, i32, P, P, P, P, P, P, P, sz, P]
        if hasattr(L, "amc_check_trace_k"):
            L.amc_check_trace_k_workspace.restype = sz
            L.amc_check_trace_k_workspace.argtypes = [i64, i32]
            L.amc_check_trace_k.argtypes = [P, P, i64, i32, i32, P, P, P, P, P, P, sz, P]
        if hasattr(L, "amc_check_well_declared"):
            L.amc_check_well_declared_workspace.restype = sz
            L.amc_check_well_declared_workspace.argtypes = [i64]
            L.amc_check_well_declared.argtypes = [P, i32, P, P, i64, P, P, i64, P, P, P, i64, P, P, P, P, sz, P]
        if hasattr(L, "amc_check_batch_guarded"):
            L.amc_check_batch_guarded_workspace.restype = sz
            L.amc_check_batch_guarded_workspace.argtypes = [i64, i64, i64]
            L.amc_check_batch_guarded.argtypes = [P, P, P, P, P, P, i64, i64, i64, P, P, P, P, sz, P]
        if hasattr(L, "amc_check_batch"):
            L.amc_check_batch_workspace.restype = sz
            L.amc_check_batch_workspace.argtypes = [i64, i64, i64]
            L.amc_check_batch.argtypes = [P, P, P, P, P, i64, i64, P, P, P, ci, P, sz, P]
        _lib = L
    return _lib


def error_string(code: int) -> str:
    try:
        return lib().amc_error_string(code).decode()
    except RuntimeError:
        return "error"


def _p(t):
    if t is None:
        return None
    return ctypes.c_void_p(t.data_ptr())


def _stream_ptr(stream):
    if stream is None:
        stream = torch.cuda.current_stream()
    return ctypes.c_void_p(stream.cuda_stream)


def _check(rc, what):
    if rc != OK:
        raise AmcError(rc, what)


def _dev(t, dtype, name):
    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise TypeError(f"{name} must be a CUDA tensor")
    if t.dtype != dtype:
        raise TypeError(f"{name} must be {dtype}, got {t.dtype}")
    if not t.is_contiguous():
        raise ValueError(f"{name} must be contiguous")
    return t


class Workspace:
    """Grow-only device scratch buffer (256-byte aligned, from torch's allocator)."""

    def __init__(self):
        self.buf = None

    def get(self, nbytes: int, device) -> torch.Tensor:
        nbytes = max(256, int(nbytes))
        if self.buf is None or self.buf.numel() < nbytes or self.buf.device != device:
            self.buf = torch.empty(nbytes + 256, dtype=torch.uint8, device=device)
        off = (-self.buf.data_ptr()) % 256
        return self.buf[off:off + nbytes]


_ws = Workspace()


def sync_status(stream=None) -> int:
    """Synchronise the stream and return (and clear) the device error word."""
    return lib().amc_sync_status(_stream_ptr(stream))


def trace_workspace_bytes(n_ops: int, n_vars: int, guarded: bool = False) -> int:
    L = lib()
    f = L.amc_check_guarded_trace_workspace if guarded else L.amc_check_trace_workspace
    return int(f(n_ops, n_vars))


TRACE_PATHS = ("scan", "small", "warp_dense", "dense", "prefix", "epochs")


def trace_plan(n_ops, n_vars, has_init=False):
    """(path name, kernels launched) of the next check_trace of these sizes
    (amc_check_trace_plan): the timed choice for the size class if one was
    made in this process, else the size rule."""
    path, launches = ctypes.c_int32(-1), ctypes.c_int32(0)
    rc = lib().amc_check_trace_plan(int(n_ops), int(n_vars), 1 if has_init else 0, ctypes.byref(path),
                                    ctypes.byref(launches))
    _check(rc, "amc_check_trace_plan")
    return TRACE_PATHS[path.value], int(launches.value)


def check_trace(kind_side, var, n_vars, init_status=None, *, guarded=False, out=None,
                workspace=None, stream=None):
    """Check one trace on the GPU (amc_check_trace / amc_check_guarded_trace).

    kind_side: uint8 CUDA tensor [n_ops]; var: int32 CUDA tensor [n_ops].
    Returns dict(step_status, final_status, var_first_fault, first_fault) of
    CUDA tensors (first_fault: int64 [1]).  ``out`` may pass preallocated
    output tensors with those keys.
    """
    _dev(kind_side, torch.uint8, "kind_side")
    _dev(var, torch.int32, "var")
    n = kind_side.numel()
    if var.numel() != n:
        raise ValueError("kind_side and var differ in length")
    dev = kind_side.device
    if init_status is not None:
        _dev(init_status, torch.uint8, "init_status")
    if out is None:
        out = dict(step_status=torch.empty(n, dtype=torch.uint8, device=dev),
                   final_status=torch.empty(max(n_vars, 0), dtype=torch.uint8, device=dev),
                   var_first_fault=torch.empty(max(n_vars, 0), dtype=torch.int32, device=dev),
                   first_fault=torch.empty(1, dtype=torch.int64, device=dev))
    nbytes = trace_workspace_bytes(n, n_vars, guarded)
    ws = workspace if workspace is not None else _ws.get(nbytes, dev)
    L = lib()
    fn = L.amc_check_guarded_trace if guarded else L.amc_check_trace
    rc = fn(_p(kind_side), _p(var), n, n_vars, _p(init_status), _p(out["step_status"]),
            _p(out["final_status"]), _p(out["var_first_fault"]), _p(out["first_fault"]),
            _p(ws), ws.numel(), _stream_ptr(stream))
    _check(rc, "amc_check_trace")
    return out


def vectorpu_overlap_pairs(arr_start, arr_len, arr_born=None, arr_died=None, n_calls=0, *, out=None, stream=None):
    """Overlap-list entries of the arrays for a run of n_calls calls (one per
    time bucket each overlapping pair's lifetimes share, both directions; every
    overlapping pair when the lifetimes are left out): the max_pairs
    translate_vectorpu_lifetimes needs (amc_vectorpu_overlap_pairs).  Returns
    the device int64 [1] tensor (``out`` if given); read it with .item()."""
    _dev(arr_start, torch.int32, "arr_start")
    _dev(arr_len, torch.int32, "arr_len")
    if (arr_born is None) != (arr_died is None):
        raise ValueError("arr_born and arr_died go together")
    if arr_born is not None:
        _dev(arr_born, torch.int32, "arr_born")
        _dev(arr_died, torch.int32, "arr_died")
    A = arr_start.numel()
    dev = arr_start.device
    L = lib()
    n = out if out is not None else torch.empty(1, dtype=torch.int64, device=dev)
    ws = _ws.get(L.amc_vectorpu_overlap_pairs_workspace(A, int(n_calls)), dev)
    rc = L.amc_vectorpu_overlap_pairs(_p(arr_start), _p(arr_len), _p(arr_born), _p(arr_died), A, int(n_calls), _p(n),
                                      _p(ws), ws.numel(), _stream_ptr(stream))
    _check(rc, "amc_vectorpu_overlap_pairs")
    return n


def translate_vectorpu_lifetimes(arr_start, arr_len, arr_parent, arr_born, arr_died, call_side, call_off,
                                 opnd_array, opnd_mode, *, infer_overlap=True, max_pairs=None, out_cap=None,
                                 known_n=None, out=None, stream=None):
    """Translate VectorPU calls over pvectors with lifetimes
    (amc_translate_vectorpu_lifetimes).  All inputs are CUDA tensors.  Returns
    dict(kind_side, var, call_first_op, arr_probe, n, n_dev, max_pairs).
    max_pairs None: counted first (amc_vectorpu_overlap_pairs, one host read).
    known_n / out: as translate_vectorpu (no host read when max_pairs is
    given too)."""
    for t, dt, nm in ((arr_start, torch.int32, "arr_start"), (arr_len, torch.int32, "arr_len"),
                      (arr_parent, torch.int32, "arr_parent"), (arr_born, torch.int32, "arr_born"),
                      (arr_died, torch.int32, "arr_died"), (call_side, torch.uint8, "call_side"),
                      (call_off, torch.int32, "call_off"), (opnd_array, torch.int32, "opnd_array"),
                      (opnd_mode, torch.uint8, "opnd_mode")):
        _dev(t, dt, nm)
    A = arr_start.numel()
    n_calls = call_side.numel()
    n_opnd = opnd_array.numel()
    dev = arr_start.device
    L = lib()
    if max_pairs is None:
        max_pairs = int(vectorpu_overlap_pairs(arr_start, arr_len, arr_born, arr_died, n_calls,
                                               stream=stream).item())
    max_pairs = max(int(max_pairs), 1)
    ws = _ws.get(L.amc_translate_vectorpu_lifetimes_workspace(A, n_calls, n_opnd, max_pairs), dev)

    def call(ks, var, cap, n_dev, first, probe):
        rc = L.amc_translate_vectorpu_lifetimes(_p(arr_start), _p(arr_len), _p(arr_parent), _p(arr_born),
                                                _p(arr_died), A, _p(call_side), _p(call_off), n_calls,
                                                _p(opnd_array), _p(opnd_mode), n_opnd, int(bool(infer_overlap)),
                                                max_pairs, _p(ks), _p(var), cap, _p(n_dev), _p(first), _p(probe),
                                                _p(ws), ws.numel(), _stream_ptr(stream))
        _check(rc, "amc_translate_vectorpu_lifetimes")

    if known_n is not None:
        n = int(known_n)
        if out is None:
            out = dict(kind_side=torch.empty(max(n, 1), dtype=torch.uint8, device=dev),
                       var=torch.empty(max(n, 1), dtype=torch.int32, device=dev),
                       call_first_op=torch.empty(n_calls + 1, dtype=torch.int64, device=dev),
                       arr_probe=torch.empty(max(A, 1), dtype=torch.int64, device=dev),
                       n_dev=torch.empty(1, dtype=torch.int64, device=dev))
        call(out["kind_side"], out["var"], n, out["n_dev"], out["call_first_op"], out["arr_probe"])
        return dict(kind_side=out["kind_side"][:n], var=out["var"][:n], call_first_op=out["call_first_op"],
                    arr_probe=out["arr_probe"][:A], n=n, n_dev=out["n_dev"], max_pairs=max_pairs)
    if out_cap is None:
        out_cap = 48 * n_calls + 2 * A + 64
    first = torch.empty(n_calls + 1, dtype=torch.int64, device=dev)
    probe = torch.empty(max(A, 1), dtype=torch.int64, device=dev)
    out_n = torch.empty(1, dtype=torch.int64, device=dev)
    for attempt in range(2):
        ks = torch.empty(max(out_cap, 1), dtype=torch.uint8, device=dev)
        var = torch.empty(max(out_cap, 1), dtype=torch.int32, device=dev)
        call(ks, var, out_cap, out_n, first, probe)
        n = int(out_n.item())
        if n <= out_cap:
            return dict(kind_side=ks[:n], var=var[:n], call_first_op=first, arr_probe=probe[:A], n=n, n_dev=out_n,
                        max_pairs=max_pairs)
        code = sync_status(stream)
        if code not in (OK, E_RANGE):
            raise AmcError(code, "amc_translate_vectorpu_lifetimes")
        out_cap = n
    raise AmcError(E_RANGE, "amc_translate_vectorpu_lifetimes")


def check_inherited_trace(kind_side, var, n_arrays, arr_parent, arr_probe, *, out=None, workspace=None,
                          stream=None):
    """Check a translated trace with creation records over 2 * n_arrays
    variables, pvectors starting from their vectors' statuses at creation
    (amc_check_inherited_trace).  Returns dict(step_status, final_status,
    var_first_fault, first_fault) of CUDA tensors."""
    _dev(kind_side, torch.uint8, "kind_side")
    _dev(var, torch.int32, "var")
    _dev(arr_parent, torch.int32, "arr_parent")
    _dev(arr_probe, torch.int64, "arr_probe")
    n = kind_side.numel()
    if var.numel() != n:
        raise ValueError("kind_side and var differ in length")
    dev = kind_side.device
    nv = 2 * n_arrays
    if out is None:
        out = dict(step_status=torch.empty(max(n, 1), dtype=torch.uint8, device=dev),
                   final_status=torch.empty(max(nv, 1), dtype=torch.uint8, device=dev),
                   var_first_fault=torch.empty(max(nv, 1), dtype=torch.int32, device=dev),
                   first_fault=torch.empty(1, dtype=torch.int64, device=dev))
    L = lib()
    ws = workspace if workspace is not None else _ws.get(L.amc_check_inherited_trace_workspace(n, n_arrays), dev)
    rc = L.amc_check_inherited_trace(_p(kind_side), _p(var), n, n_arrays, _p(arr_parent), _p(arr_probe),
                                     _p(out["step_status"]), _p(out["final_status"]), _p(out["var_first_fault"]),
                                     _p(out["first_fault"]), _p(ws), ws.numel(), _stream_ptr(stream))
    _check(rc, "amc_check_inherited_trace")
    return dict(step_status=out["step_status"][:n], final_status=out["final_status"][:nv],
                var_first_fault=out["var_first_fault"][:nv], first_fault=out["first_fault"])


def check_trace_k(op, var, n_vars, k, init_status=None, *, out=None, workspace=None, stream=None):
    """Trace check over k memory locations (amc_check_trace_k).  op uint8 /
    var int32 CUDA tensors; statuses are bit masks of valid locations, 0x80 =
    stuck.  Returns dict(step_status, final_status, var_first_fault,
    first_fault)."""
    _dev(op, torch.uint8, "op")
    _dev(var, torch.int32, "var")
    n = op.numel()
    dev = op.device
    if init_status is not None:
        _dev(init_status, torch.uint8, "init_status")
    if out is None:
        out = dict(step_status=torch.empty(n, dtype=torch.uint8, device=dev),
                   final_status=torch.empty(max(n_vars, 0), dtype=torch.uint8, device=dev),
                   var_first_fault=torch.empty(max(n_vars, 0), dtype=torch.int32, device=dev),
                   first_fault=torch.empty(1, dtype=torch.int64, device=dev))
    L = lib()
    ws = workspace if workspace is not None else _ws.get(L.amc_check_trace_k_workspace(n, n_vars), dev)
    rc = L.amc_check_trace_k(_p(op), _p(var), n, n_vars, k, _p(init_status), _p(out["step_status"]),
                             _p(out["final_status"]), _p(out["var_first_fault"]), _p(out["first_fault"]), _p(ws),
                             ws.numel(), _stream_ptr(stream))
    _check(rc, "amc_check_trace_k")
    return out


def _host(t, dtype, name):
    if not isinstance(t, torch.Tensor) or t.device.type != "cpu":
        raise TypeError(f"{name} must be a CPU tensor")
    if t.dtype != dtype:
        raise TypeError(f"{name} must be {dtype}, got {t.dtype}")
    if not t.is_contiguous():
        raise ValueError(f"{name} must be contiguous")
    return t


def check_trace_host(kind_side, var, n_vars, init_status=None, *, chunk_ops=0, out=None, workspace=None,
                     stream=None, device=None):
    """Check one trace held in host memory (amc_check_trace_host): the library
    copies it in chunk by chunk, checks each chunk on the GPU and copies the
    step statuses back while the next chunk is on its way.

    kind_side: uint8 CPU tensor [n_ops]; var: int32 CPU tensor [n_ops];
    init_status: uint8 CPU tensor [n_vars] or None.  Pinned tensors
    (``pin_memory=True``) let the copies overlap the checks.  Returns
    dict(step_status, final_status, var_first_fault, first_fault) of CPU
    tensors (pinned when allocated here), complete once ``stream`` (default:
    the current stream) has synchronised, e.g. through ``sync_status``.
    """
    _host(kind_side, torch.uint8, "kind_side")
    _host(var, torch.int32, "var")
    n = kind_side.numel()
    if var.numel() != n:
        raise ValueError("kind_side and var differ in length")
    if init_status is not None:
        _host(init_status, torch.uint8, "init_status")
        if init_status.numel() != n_vars:
            raise ValueError("init_status must hold n_vars statuses")
    dev = torch.device("cuda", torch.cuda.current_device()) if device is None else torch.device(device)
    if out is None:
        out = dict(step_status=torch.empty(n, dtype=torch.uint8, pin_memory=True),
                   final_status=torch.empty(max(n_vars, 0), dtype=torch.uint8, pin_memory=True),
                   var_first_fault=torch.empty(max(n_vars, 0), dtype=torch.int32, pin_memory=True),
                   first_fault=torch.empty(1, dtype=torch.int64, pin_memory=True))
    L = lib()
    nbytes = int(L.amc_check_trace_host_workspace(n, n_vars, int(chunk_ops)))
    ws = workspace if workspace is not None else _ws.get(nbytes, dev)
    rc = L.amc_check_trace_host(_p(kind_side), _p(var), n, n_vars, _p(init_status), _p(out["step_status"]),
                                _p(out["final_status"]), _p(out["var_first_fault"]), _p(out["first_fault"]),
                                int(chunk_ops), _p(ws), ws.numel(), _stream_ptr(stream))
    _check(rc, "amc_check_trace_host")
    return out


def trace_host_workspace_bytes(n_ops: int, n_vars: int, chunk_ops: int = 0) -> int:
    return int(lib().amc_check_trace_host_workspace(n_ops, n_vars, chunk_ops))


def translate_vectorpu(arr_start, arr_len, call_side, call_off, opnd_array, opnd_mode, *,
                       infer_overlap=True, out_cap=None, known_n=None, out=None, stream=None):
    """Translate VectorPU calls into a core trace over 2 * n_arrays variables
    (amc_translate_vectorpu).  All inputs are CUDA tensors (int32 / uint8).
    Returns dict(kind_side, var, call_first_op, n, n_dev).  When ``out_cap`` is
    too small the call is repeated once with the exact size.

    ``known_n``: the statement count of an earlier translation of the same
    calls; the call then reads nothing back (no host synchronisation) and
    returns the outputs cut to known_n statements (``out`` may pass tensors
    from an earlier call's result to reuse); a different count is reported by
    sync_status (E_RANGE when larger)."""
    _dev(arr_start, torch.int32, "arr_start")
    _dev(arr_len, torch.int32, "arr_len")
    _dev(call_side, torch.uint8, "call_side")
    _dev(call_off, torch.int32, "call_off")
    _dev(opnd_array, torch.int32, "opnd_array")
    _dev(opnd_mode, torch.uint8, "opnd_mode")
    A = arr_start.numel()
    n_calls = call_side.numel()
    n_opnd = opnd_array.numel()
    dev = arr_start.device
    L = lib()
    if known_n is not None:
        n = int(known_n)
        if out is None:
            out = dict(kind_side=torch.empty(max(n, 1), dtype=torch.uint8, device=dev),
                       var=torch.empty(max(n, 1), dtype=torch.int32, device=dev),
                       call_first_op=torch.empty(n_calls + 1, dtype=torch.int64, device=dev),
                       n_dev=torch.empty(1, dtype=torch.int64, device=dev))
        ws = _ws.get(L.amc_translate_vectorpu_workspace(A, n_calls, n_opnd), dev)
        rc = L.amc_translate_vectorpu(_p(arr_start), _p(arr_len), A, _p(call_side), _p(call_off), n_calls,
                                      _p(opnd_array), _p(opnd_mode), n_opnd, int(bool(infer_overlap)),
                                      _p(out["kind_side"]), _p(out["var"]), n, _p(out["n_dev"]),
                                      _p(out["call_first_op"]), _p(ws), ws.numel(), _stream_ptr(stream))
        _check(rc, "amc_translate_vectorpu")
        return dict(kind_side=out["kind_side"][:n], var=out["var"][:n], call_first_op=out["call_first_op"], n=n,
                    n_dev=out["n_dev"])
    if out_cap is None:
        out_cap = 48 * n_calls + 64
    first = torch.empty(n_calls + 1, dtype=torch.int64, device=dev)
    out_n = torch.empty(1, dtype=torch.int64, device=dev)
    ws = _ws.get(L.amc_translate_vectorpu_workspace(A, n_calls, n_opnd), dev)
    for attempt in range(2):
        ks = torch.empty(max(out_cap, 1), dtype=torch.uint8, device=dev)
        var = torch.empty(max(out_cap, 1), dtype=torch.int32, device=dev)
        rc = L.amc_translate_vectorpu(_p(arr_start), _p(arr_len), A, _p(call_side), _p(call_off), n_calls,
                                      _p(opnd_array), _p(opnd_mode), n_opnd, int(bool(infer_overlap)),
                                      _p(ks), _p(var), out_cap, _p(out_n), _p(first), _p(ws), ws.numel(),
                                      _stream_ptr(stream))
        _check(rc, "amc_translate_vectorpu")
        n = int(out_n.item())
        if n <= out_cap:
            return dict(kind_side=ks[:n], var=var[:n], call_first_op=first, n=n, n_dev=out_n)
        code = sync_status(stream)
        if code not in (OK, E_RANGE):
            raise AmcError(code, "amc_translate_vectorpu")
        out_cap = n
    raise AmcError(E_RANGE, "amc_translate_vectorpu")


def check_batch(tok, payload, prog_tok_off, prog_nvars, prog_var_off=None, *, graph_capture=False, out=None,
                workspace=None, stream=None):
    """Relation-mode check of a batch of programs (amc_check_batch).

    tok uint8 [T], payload int32 [T], prog_tok_off int64 [P+1], prog_nvars
    int32 [P], prog_var_off int64 [P+1] (computed from prog_nvars if None), all
    CUDA tensors.  Returns dict(step_mask, final_mask, prog_first_fault)."""
    _dev(tok, torch.uint8, "tok")
    _dev(payload, torch.int32, "payload")
    _dev(prog_tok_off, torch.int64, "prog_tok_off")
    _dev(prog_nvars, torch.int32, "prog_nvars")
    dev = tok.device
    P = prog_nvars.numel()
    if prog_var_off is None:
        prog_var_off = torch.zeros(P + 1, dtype=torch.int64, device=dev)
        torch.cumsum(prog_nvars.to(torch.int64), 0, out=prog_var_off[1:])
    _dev(prog_var_off, torch.int64, "prog_var_off")
    n_tok = tok.numel()
    total_vars = int(prog_var_off[-1].item()) if P > 0 else 0
    if out is None:
        out = dict(step_mask=torch.empty(n_tok, dtype=torch.uint8, device=dev),
                   final_mask=torch.empty(total_vars, dtype=torch.uint8, device=dev),
                   prog_first_fault=torch.empty(P, dtype=torch.int64, device=dev))
    L = lib()
    nbytes = L.amc_check_batch_workspace(n_tok, P, total_vars)
    ws = workspace if workspace is not None else _ws.get(nbytes, dev)
    rc = L.amc_check_batch(_p(tok), _p(payload), _p(prog_tok_off), _p(prog_nvars), _p(prog_var_off), P, n_tok,
                           _p(out["step_mask"]), _p(out["final_mask"]), _p(out["prog_first_fault"]),
                           int(bool(graph_capture)), _p(ws), ws.numel(), _stream_ptr(stream))
    _check(rc, "amc_check_batch")
    return out


def check_batch_guarded(tok, payload, prog_tok_off, prog_nvars, prog_guard, prog_var_off=None, *, out=None,
                        workspace=None, stream=None):
    """Path-sensitive relation mode over a batch (amc_check_batch_guarded):
    IF / WHILE bits 4-5 = condition (0 opaque, 1 isValid g, 2 remIsValid g)
    on each program's guard variable prog_guard[p] (int32, -1 none).  Other
    arguments and the returned dict as check_batch."""
    _dev(tok, torch.uint8, "tok")
    _dev(payload, torch.int32, "payload")
    _dev(prog_tok_off, torch.int64, "prog_tok_off")
    _dev(prog_nvars, torch.int32, "prog_nvars")
    _dev(prog_guard, torch.int32, "prog_guard")
    dev = tok.device
    P = prog_nvars.numel()
    if prog_var_off is None:
        prog_var_off = torch.zeros(P + 1, dtype=torch.int64, device=dev)
        torch.cumsum(prog_nvars.to(torch.int64), 0, out=prog_var_off[1:])
    _dev(prog_var_off, torch.int64, "prog_var_off")
    n_tok = tok.numel()
    total_vars = int(prog_var_off[-1].item()) if P > 0 else 0
    if out is None:
        out = dict(step_mask=torch.empty(n_tok, dtype=torch.uint8, device=dev),
                   final_mask=torch.empty(total_vars, dtype=torch.uint8, device=dev),
                   prog_first_fault=torch.empty(P, dtype=torch.int64, device=dev))
    L = lib()
    nbytes = L.amc_check_batch_guarded_workspace(n_tok, P, total_vars)
    ws = workspace if workspace is not None else _ws.get(nbytes, dev)
    rc = L.amc_check_batch_guarded(_p(tok), _p(payload), _p(prog_tok_off), _p(prog_nvars), _p(prog_var_off),
                                   _p(prog_guard), P, n_tok, total_vars, _p(out["step_mask"]), _p(out["final_mask"]),
                                   _p(out["prog_first_fault"]), _p(ws), ws.numel(), _stream_ptr(stream))
    _check(rc, "amc_check_batch_guarded")
    return out


def check_well_declared(arr_loc_off, loc_owner, call_tok_off, tok, payload, call_am_off, am_array, am_mode, *,
                        out=None, stream=None):
    """Static well-declaredness of calls AM{S} (amc_check_well_declared).

    arr_loc_off int64 [A+1], loc_owner int32 [locations], call_tok_off int64
    [C+1], tok uint8 / payload int32 [T], call_am_off int64 [C+1], am_array
    int32 / am_mode uint8 [D], all CUDA tensors.  Returns dict(violations
    uint32 -> int32 view, first_bad int64, first_unmet int32)."""
    _dev(arr_loc_off, torch.int64, "arr_loc_off")
    _dev(loc_owner, torch.int32, "loc_owner")
    _dev(call_tok_off, torch.int64, "call_tok_off")
    _dev(tok, torch.uint8, "tok")
    _dev(payload, torch.int32, "payload")
    _dev(call_am_off, torch.int64, "call_am_off")
    _dev(am_array, torch.int32, "am_array")
    _dev(am_mode, torch.uint8, "am_mode")
    dev = tok.device
    C = call_tok_off.numel() - 1
    if out is None:
        out = dict(violations=torch.empty(C, dtype=torch.int32, device=dev),
                   first_bad=torch.empty(C, dtype=torch.int64, device=dev),
                   first_unmet=torch.empty(C, dtype=torch.int32, device=dev))
    L = lib()
    ws = _ws.get(L.amc_check_well_declared_workspace(C), dev)
    rc = L.amc_check_well_declared(_p(arr_loc_off), arr_loc_off.numel() - 1, _p(loc_owner), _p(call_tok_off), C,
                                   _p(tok), _p(payload), tok.numel(), _p(call_am_off), _p(am_array), _p(am_mode),
                                   am_array.numel(), _p(out["violations"]), _p(out["first_bad"]),
                                   _p(out["first_unmet"]), _p(ws), ws.numel(), _stream_ptr(stream))
    _check(rc, "amc_check_well_declared")
    return out


# --------------------------------------------------------------------------
# Serving
# --------------------------------------------------------------------------
REQ_TRACE, REQ_PROGRAM = 0, 1


class _Request(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int), ("n_vars", ctypes.c_int32), ("n_items", ctypes.c_int64),
                ("kind_side", ctypes.c_void_p), ("var", ctypes.c_void_p), ("flags", ctypes.c_int)]


class _Result(ctypes.Structure):
    _fields_ = [("error", ctypes.c_int), ("first_fault", ctypes.c_int64), ("n_items", ctypes.c_int64),
                ("status", ctypes.c_void_p), ("t_submit", ctypes.c_double), ("t_admit", ctypes.c_double),
                ("t_done", ctypes.c_double), ("is_mask", ctypes.c_int)]


class Server:
    """Continuous-batching check server (amc_server_create / amc_serve_*).

    Requests are numpy arrays on the host: op bytes (uint8) and var ids
    (int32) for traces; token bytes and payloads for programs.  A session's
    variable status sets stay on the device between its requests, which may
    be of either kind."""

    def __init__(self, mem_budget_bytes: int = 32 << 30, max_slots: int = 16):
        import numpy as np  # noqa: F401
        L = lib()
        P = ctypes.c_void_p
        L.amc_server_create.argtypes = [ctypes.c_size_t, ctypes.c_int, ctypes.POINTER(P)]
        L.amc_serve_submit.argtypes = [P, ctypes.c_uint64, ctypes.POINTER(_Request), ctypes.POINTER(ctypes.c_uint64)]
        L.amc_serve_poll.argtypes = [P, ctypes.c_uint64, ctypes.POINTER(ctypes.c_int), ctypes.POINTER(_Result)]
        L.amc_serve_release.argtypes = [P, ctypes.c_uint64]
        L.amc_serve_completed.argtypes = [P, P, ctypes.c_int32, ctypes.POINTER(ctypes.c_int32)]
        L.amc_session_export.argtypes = [P, ctypes.c_uint64, P, ctypes.c_int32]
        L.amc_server_destroy.argtypes = [P]
        self._L = L
        self._h = P()
        _check(L.amc_server_create(mem_budget_bytes, max_slots, ctypes.byref(self._h)), "amc_server_create")

    def submit(self, session: int, kind: int, n_vars: int, kind_side, var, borrow: bool = False):
        """Queue a request; returns its ticket, or None when the server pushes back.

        kind_side / var: numpy arrays or CPU tensors.  borrow=True: the server
        reads them when the request runs instead of copying them now; the
        caller keeps them alive and unchanged until poll() reports the request
        done (pinned tensors make the copy asynchronous)."""
        import numpy as np
        if isinstance(kind_side, torch.Tensor):
            ks, v = kind_side, var
            if ks.dtype != torch.uint8 or v.dtype != torch.int32 or not (ks.is_contiguous() and v.is_contiguous()):
                raise TypeError("kind_side / var must be contiguous uint8 / int32 tensors")
            n, pk, pv = ks.numel(), ks.data_ptr(), v.data_ptr()
        else:
            ks = np.ascontiguousarray(kind_side, dtype=np.uint8)
            v = np.ascontiguousarray(var, dtype=np.int32)
            n, pk, pv = ks.shape[0], ks.ctypes.data, v.ctypes.data
        req = _Request(kind, n_vars, n, pk, pv, 1 if borrow else 0)
        t = ctypes.c_uint64()
        rc = self._L.amc_serve_submit(self._h, session, ctypes.byref(req), ctypes.byref(t))
        if rc == E_AGAIN:
            return None
        _check(rc, "amc_serve_submit")
        return t.value

    def poll(self, ticket: int, release: bool = True):
        """None while running; else dict(status, is_mask, first_fault, error, t_submit, t_admit, t_done)."""
        import numpy as np
        done = ctypes.c_int()
        res = _Result()
        _check(self._L.amc_serve_poll(self._h, ticket, ctypes.byref(done), ctypes.byref(res)), "amc_serve_poll")
        if not done.value:
            return None
        n = res.n_items
        status = np.ctypeslib.as_array((ctypes.c_uint8 * n).from_address(res.status)).copy() if n else \
            np.zeros(0, np.uint8)
        out = dict(status=status, is_mask=bool(res.is_mask), first_fault=res.first_fault, error=res.error,
                   t_submit=res.t_submit, t_admit=res.t_admit, t_done=res.t_done)
        if release:
            _check(self._L.amc_serve_release(self._h, ticket), "amc_serve_release")
        return out

    def completed(self, cap: int = 4096):
        """Tickets of the requests finished since the last call (amc_serve_completed)."""
        buf = (ctypes.c_uint64 * cap)()
        n = ctypes.c_int32()
        _check(self._L.amc_serve_completed(self._h, ctypes.cast(buf, ctypes.c_void_p), cap, ctypes.byref(n)),
               "amc_serve_completed")
        return list(buf[:n.value])

    def export(self, session: int, n_vars: int):
        import numpy as np
        out = np.empty(n_vars, np.uint8)
        _check(self._L.amc_session_export(self._h, session, out.ctypes.data, n_vars), "amc_session_export")
        return out

    def close(self):
        if self._h:
            _check(self._L.amc_server_destroy(self._h), "amc_server_destroy")
            self._h = ctypes.c_void_p()

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()
