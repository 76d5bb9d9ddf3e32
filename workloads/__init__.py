"""Seeded synthetic workloads for the access-mode consistency checker.

Input generation only: nothing here applies an effect, composes a transfer
function or evaluates a program.  Both the oracle tests and the CUDA path read
their inputs from these generators, so the two sides always see the same bytes.

Encodings (shared with the C ABI): op byte = kind | side << 4 with kinds
r=0 w=1 Push=2 Pull=3 Noop=4, side 0 = CPU (local), 1 = GPU (remote);
structure tokens IF=8 ELSE=9 WHILE=10 END=11; annotation modes R=1 W=2 RW=3
with bit 7 marking an annotation dropped by fault injection.

Workloads (seeds fixed by the benchmark definition):
  trace_uniform   16 vars, 4,096 ops, uniform kind / side / var         (seed 0)
  trace_zipf      2^30 ops, 2^20 vars, Zipf(1.05) ids, kind mix
                  r .40 w .20 Push .15 Pull .15 Noop .10, side 50/50     (seed 1)
  vectorpu_calls  4,096 intervals over 2^24, 2^24 calls of 1-4 operands,
                  modes R/W/RW .5/.3/.2, 1e-4 dropped                    (seed 2)
  programs        100,000 If/While programs over 64-4,096 vars           (seed 3)
  serve_requests  Poisson arrivals of trace / program requests          (seed 4)
  wd_calls        calls AM{S} for the static well-declaredness check    (seed 5)
  vectorpu_lifetimes  16 vectors of 2^20 elements, 65,536 pvectors created
                  and deleted during 2^24 calls (about 4,096 live at a time) (seed 6)
  programs_guarded  20,000 programs over 16-256 vars whose conditions test a
                  guard variable (isValid / remIsValid) or are opaque    (seed 7)
"""
from __future__ import annotations

import ctypes
import math
import os
import subprocess

import numpy as np

KIND_MIX = (0.40, 0.20, 0.15, 0.15, 0.10)          # r, w, Push, Pull, Noop
R, W, RW, DROPPED = 1, 2, 3, 0x80

_HERE = os.path.dirname(os.path.abspath(__file__))
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "libworkloads.so")
_lib = None


def build(force: bool = False) -> str:
    src = os.path.join(_HERE, "progs.c")
    if not force and os.path.exists(_LIB_PATH) and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(src):
        return _LIB_PATH
    os.makedirs(_BUILD, exist_ok=True)
    tmp = _LIB_PATH + f".tmp{os.getpid()}"
    subprocess.check_call(["gcc", "-O2", "-std=c11", "-shared", "-fPIC", "-o", tmp, src, "-lm"])
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _clib():
    global _lib
    if _lib is None:
        _lib = ctypes.CDLL(build())
        P = ctypes.c_void_p
        _lib.wl_program_sizes.argtypes = [P, P, ctypes.c_uint64, ctypes.c_int64, ctypes.c_int64, P, P, P]
        _lib.wl_program_fill.argtypes = [P, P, ctypes.c_uint64, ctypes.c_int64, ctypes.c_int64, P, P, P]
        _lib.wl_wd_sizes.argtypes = [P, ctypes.c_int32, ctypes.c_uint64, ctypes.c_int64, P, ctypes.c_double, P, P]
        _lib.wl_wd_fill.argtypes = [P, ctypes.c_int32, ctypes.c_uint64, ctypes.c_int64, P, ctypes.c_double, P, P,
                                    P, P, P, P]
        _lib.wl_lifetimes_arrays.argtypes = [ctypes.c_uint64, ctypes.c_int32, ctypes.c_int32, ctypes.c_int32,
                                             ctypes.c_int64, ctypes.c_double, ctypes.c_double, ctypes.c_double,
                                             P, P, P, P, P]
        _lib.wl_lifetimes_calls.argtypes = [ctypes.c_uint64, ctypes.c_int32, P, P, ctypes.c_int64, ctypes.c_int32, P,
                                            ctypes.c_double, P, P, P, P, P]
    return _lib


def _p(a):
    return a.ctypes.data_as(ctypes.c_void_p)


# --------------------------------------------------------------------------
# Straight-line traces
# --------------------------------------------------------------------------
def trace_uniform(seed: int = 0, n_ops: int = 4096, n_vars: int = 16):
    """Uniform kind over the five core ops, uniform side, uniform var; drawn as
    three independent ``integers`` calls in that order (numpy PCG64)."""
    rng = np.random.default_rng(seed)
    kind = rng.integers(0, 5, n_ops)
    side = rng.integers(0, 2, n_ops)
    var = rng.integers(0, n_vars, n_ops)
    ks = (kind | (side << 4)).astype(np.uint8)
    return ks, var.astype(np.int32), n_vars


def zipf_cdf(n_vars: int, s: float = 1.05) -> np.ndarray:
    k = np.arange(1, n_vars + 1, dtype=np.float64)
    w = k ** (-s)
    c = np.cumsum(w)
    return c / c[-1]


def trace_zipf(n_ops: int = 1 << 30, n_vars: int = 1 << 20, seed: int = 1, device="cpu",
               s: float = 1.05, kind_mix=KIND_MIX, chunk: int = 1 << 26):
    """Zipf(s) variable ids (rank - 1, heavy ids first, by inverse CDF), the
    given kind mix and a fair side bit.  Generated with torch on ``device``
    (Philox on CUDA), in chunks, so 2^30 ops fit in memory.  Returns torch
    tensors (kind_side uint8, var int32)."""
    import torch
    dev = torch.device(device)
    g = torch.Generator(device=dev)
    g.manual_seed(seed)
    cdf = torch.from_numpy(zipf_cdf(n_vars, s)).to(dev)
    kcdf = torch.tensor(np.cumsum(kind_mix)[:-1], dtype=torch.float64, device=dev)
    ks = torch.empty(n_ops, dtype=torch.uint8, device=dev)
    var = torch.empty(n_ops, dtype=torch.int32, device=dev)
    for lo in range(0, n_ops, chunk):
        n = min(chunk, n_ops - lo)
        u = torch.rand(n, dtype=torch.float64, device=dev, generator=g)
        v = torch.searchsorted(cdf, u).clamp_(max=n_vars - 1)
        var[lo:lo + n] = v.to(torch.int32)
        del u, v
        u = torch.rand(n, dtype=torch.float64, device=dev, generator=g)
        kind = torch.searchsorted(kcdf, u, right=True)
        del u
        side = torch.randint(0, 2, (n,), device=dev, generator=g)
        ks[lo:lo + n] = (kind | (side << 4)).to(torch.uint8)
        del kind, side
    return ks, var


def trace_random(rng: np.random.Generator, n_ops: int, n_vars: int, kinds=(0, 1, 2, 3, 4),
                 p=None, zipf_s: float | None = None):
    """Small random traces for tests (numpy)."""
    kind = rng.choice(np.asarray(kinds), size=n_ops, p=p)
    side = rng.integers(0, 2, n_ops)
    if zipf_s is None:
        var = rng.integers(0, n_vars, n_ops)
    else:
        var = np.searchsorted(zipf_cdf(n_vars, zipf_s), rng.random(n_ops))
        var = np.minimum(var, n_vars - 1)
    return (kind | (side << 4)).astype(np.uint8), var.astype(np.int32)


# --------------------------------------------------------------------------
# VectorPU calls over overlapping intervals
# --------------------------------------------------------------------------
def vectorpu_calls(seed: int = 2, n_arrays: int = 4096, space: int = 1 << 24,
                   n_calls: int = 1 << 24, len_log2=(8.0, 16.0), max_opnds: int = 4,
                   mode_p=(0.5, 0.3, 0.2), drop_p: float = 1e-4):
    """Intervals [start, start + len) with start uniform in [0, space), len =
    floor(2^U(a, b)) clipped to the space; calls with a fair side bit, 1..max
    distinct operands drawn uniformly, modes R/W/RW and dropped annotations."""
    rng = np.random.default_rng(seed)
    start = rng.integers(0, space, n_arrays)
    length = np.floor(2.0 ** rng.uniform(len_log2[0], len_log2[1], n_arrays)).astype(np.int64)
    length = np.maximum(1, np.minimum(length, space - start))
    side = rng.integers(0, 2, n_calls).astype(np.uint8)
    cnt = rng.integers(1, max_opnds + 1, n_calls)
    max_opnds = min(max_opnds, n_arrays)
    cnt = np.minimum(cnt, n_arrays)
    cand = rng.integers(0, n_arrays, (n_calls, max_opnds))
    # redraw collisions until the first cnt entries of each call are distinct
    while True:
        dup = np.zeros((n_calls, max_opnds), bool)
        for j in range(1, max_opnds):
            for i in range(j):
                dup[:, j] |= cand[:, j] == cand[:, i]
        dup &= np.arange(max_opnds)[None, :] < cnt[:, None]
        nd = int(dup.sum())
        if nd == 0:
            break
        cand[dup] = rng.integers(0, n_arrays, nd)
    mask = np.arange(max_opnds)[None, :] < cnt[:, None]
    opnd_array = cand[mask].astype(np.int32)
    n_op = opnd_array.shape[0]
    mode = (rng.choice(np.array([R, W, RW]), size=n_op, p=mode_p)).astype(np.uint8)
    drop = rng.random(n_op) < drop_p
    mode[drop] |= DROPPED
    call_off = np.zeros(n_calls + 1, np.int64)
    np.cumsum(cnt, out=call_off[1:])
    return dict(arr_start=start.astype(np.int32), arr_len=length.astype(np.int32),
                call_side=side, call_off=call_off.astype(np.int32),
                opnd_array=opnd_array, opnd_mode=mode)


# --------------------------------------------------------------------------
# Structured programs
# --------------------------------------------------------------------------
def _prog_params(p_if=0.05, p_while=0.03, max_depth=4, max_branch=32, max_body=64,
                 median=2048.0, sigma=0.7356, max_len=1 << 20, vars_lo=64, vars_hi=4096,
                 kind_mix=KIND_MIX):
    cdf = np.cumsum(kind_mix)
    dp = np.array([p_if, p_while, median, sigma, *cdf], np.float64)
    ip = np.array([max_depth, max_branch, max_body, max_len, vars_lo, vars_hi], np.int64)
    return dp, ip


def programs(n_progs: int = 100_000, seed: int = 3, first: int = 0, **kw):
    """Batch of programs: n_vars uniform in [vars_lo, vars_hi]; leaf-op count
    clip(round(lognormal(ln median, sigma)), 1, max_len); at each node of depth
    < max_depth an If (p_if; then/else get uniform 0..max_branch leaf ops) or a
    While (p_while; body of uniform 1..max_body leaf ops), otherwise an op with
    the kind mix, a fair side and a uniform program-local var."""
    dp, ip = _prog_params(**kw)
    lib = _clib()
    n_tok = np.empty(n_progs, np.int64)
    n_vars = np.empty(n_progs, np.int32)
    n_leaf = np.empty(n_progs, np.int64)
    lib.wl_program_sizes(_p(dp), _p(ip), seed, first, n_progs, _p(n_tok), _p(n_vars), _p(n_leaf))
    tok_off = np.zeros(n_progs + 1, np.int64)
    np.cumsum(n_tok, out=tok_off[1:])
    tok = np.empty(int(tok_off[-1]), np.uint8)
    payload = np.empty(int(tok_off[-1]), np.int32)
    lib.wl_program_fill(_p(dp), _p(ip), seed, first, n_progs, _p(tok_off), _p(tok), _p(payload))
    return dict(tok=tok, payload=payload, prog_tok_off=tok_off, prog_nvars=n_vars,
                n_leaf=n_leaf)


# --------------------------------------------------------------------------
# Calls AM{S} for the static well-declaredness check
# --------------------------------------------------------------------------
def programs_guarded(n_progs: int = 20_000, seed: int = 7, p_cond=(1 / 3, 1 / 3, 1 / 3), **kw):
    """Structured programs (programs(), seed 7, 16-256 variables and a median
    of 2,000 tokens unless given) with a guard variable g drawn uniformly per
    program: each If's condition is drawn from opaque / isValid g /
    remIsValid g with probabilities p_cond (bits 4-5 of the token); Whiles
    keep opaque conditions (a While on g whose body leaves g alone would never
    end); the ops on g become writes or Noops (kind w .7 / Noop .3, side
    unchanged), so that g flips between its sides and is never stuck.
    Returns the dict of programs() plus prog_guard (int32)."""
    kw.setdefault("vars_lo", 16)
    kw.setdefault("vars_hi", 256)
    kw.setdefault("median", 2000.0)
    b = programs(n_progs, seed=seed, **kw)
    rng = np.random.default_rng(seed)
    tok, pay, off = b["tok"], b["payload"], b["prog_tok_off"]
    nv = b["prog_nvars"].astype(np.int64)
    guard = np.floor(rng.random(nv.size) * nv).astype(np.int32)
    k = tok & 15
    ifs = np.nonzero(k == 8)[0]
    c = rng.choice(3, size=ifs.size, p=np.asarray(p_cond, np.float64))
    tok[ifs] = (tok[ifs] & 15) | (c.astype(np.uint8) << 4)
    prog_of = np.repeat(np.arange(nv.size), np.diff(off))
    on_g = np.nonzero((k <= 4) & (pay == guard[prog_of]))[0]
    kind = np.where(rng.random(on_g.size) < 0.7, 1, 4).astype(np.uint8)
    tok[on_g] = (tok[on_g] & 0x10) | kind
    b["prog_guard"] = guard
    return b


def wd_calls(n_calls: int = 1 << 20, n_arrays: int = 4096, len_range=(1, 64), seed: int = 5,
             mode_p=(0.5, 0.3, 0.2), p_bad: float = 0.01):
    """Arrays of len_range locations (uniform); per call one side, 1..4
    declarations on distinct arrays (modes R / W / RW with mode_p) and a body
    built from them (every location of a W array written, at top level or in
    both branches of an If; 1..4 reads for R, reads and writes for RW, some in
    a While; Noops); with probability p_bad one injected flaw (a W array
    written in one branch or in a While only, an undeclared access, a read of
    a W array, a Push).  Returns the CSR arrays of oracle.well_declared."""
    rng = np.random.default_rng(seed)
    lens = rng.integers(len_range[0], len_range[1] + 1, n_arrays)
    a_off = np.zeros(n_arrays + 1, np.int64)
    np.cumsum(lens, out=a_off[1:])
    owner = np.repeat(np.arange(n_arrays, dtype=np.int32), lens)
    pm = np.array(mode_p, np.float64)
    lib = _clib()
    n_tok = np.empty(n_calls, np.int64)
    n_decl = np.empty(n_calls, np.int32)
    lib.wl_wd_sizes(_p(a_off), n_arrays, seed, n_calls, _p(pm), p_bad, _p(n_tok), _p(n_decl))
    tok_off = np.zeros(n_calls + 1, np.int64)
    np.cumsum(n_tok, out=tok_off[1:])
    am_off = np.zeros(n_calls + 1, np.int64)
    np.cumsum(n_decl, out=am_off[1:])
    tok = np.empty(int(tok_off[-1]), np.uint8)
    payload = np.empty(int(tok_off[-1]), np.int32)
    am_array = np.empty(int(am_off[-1]), np.int32)
    am_mode = np.empty(int(am_off[-1]), np.uint8)
    lib.wl_wd_fill(_p(a_off), n_arrays, seed, n_calls, _p(pm), p_bad, _p(tok_off), _p(am_off), _p(tok), _p(payload),
                   _p(am_array), _p(am_mode))
    return dict(arr_loc_off=a_off, loc_owner=owner, call_tok_off=tok_off, tok=tok, payload=payload,
                call_am_off=am_off, am_array=am_array, am_mode=am_mode)


def vectorpu_lifetimes(seed: int = 6, n_vectors: int = 16, vec_len: int = 1 << 20, n_pvectors: int = 65536,
                       n_calls: int = 1 << 24, len_log2=(8.0, 16.0), mean_life: float | None = None,
                       max_opnds: int = 4, mode_p=(0.5, 0.3, 0.2), drop_p: float = 1e-4):
    """VectorPU calls over pvectors that are created and deleted during the
    run: n_vectors vectors of vec_len elements side by side (ids 0..), live
    throughout; n_pvectors pvectors (ids after them), each a sub-range of a
    uniformly drawn vector (start uniform in it, length floor(2^U(a, b))
    clipped to its end), created before a uniform call and live for an
    exponential number of calls of mean mean_life (default n_calls / 16, so
    that about n_pvectors / 16 are live at a time); calls with a fair side and
    1..max_opnds distinct operands drawn from the arrays live at the call,
    modes R / W / RW with mode_p, annotations dropped with drop_p.  Returns
    the inputs of oracle.vectorpu_lifetimes."""
    A = n_vectors + n_pvectors
    life = float(n_calls) / 16.0 if mean_life is None else float(mean_life)
    lib = _clib()
    start = np.empty(A, np.int32)
    length = np.empty(A, np.int32)
    parent = np.empty(A, np.int32)
    born = np.empty(A, np.int32)
    died = np.empty(A, np.int32)
    lib.wl_lifetimes_arrays(seed, n_vectors, vec_len, A, n_calls, len_log2[0], len_log2[1], life, _p(start),
                            _p(length), _p(parent), _p(born), _p(died))
    side = np.empty(n_calls, np.uint8)
    cnt = np.empty(n_calls, np.int32)
    pm = np.array(mode_p, np.float64)
    if lib.wl_lifetimes_calls(seed, A, _p(born), _p(died), n_calls, max_opnds, _p(pm), drop_p, _p(side), _p(cnt),
                              None, None, None) != 0:
        raise MemoryError("workload generator")
    call_off = np.zeros(n_calls + 1, np.int64)
    np.cumsum(cnt, out=call_off[1:])
    opnd_array = np.empty(int(call_off[-1]), np.int32)
    opnd_mode = np.empty(int(call_off[-1]), np.uint8)
    lib.wl_lifetimes_calls(seed, A, _p(born), _p(died), n_calls, max_opnds, _p(pm), drop_p, _p(side), _p(cnt),
                           _p(call_off), _p(opnd_array), _p(opnd_mode))
    return dict(arr_start=start, arr_len=length, arr_parent=parent, arr_born=born, arr_died=died, call_side=side,
                call_off=call_off.astype(np.int32), opnd_array=opnd_array, opnd_mode=opnd_mode)


# --------------------------------------------------------------------------
# Serving requests
# --------------------------------------------------------------------------
SERVE_NV_GRID = tuple(range(64, 4097, 128))        # 32 session sizes, 64 .. 4,032 variables


def serve_schedule(rate: float, n_requests: int = 10_000, seed: int = 4, trace_log2=(10.0, 24.0),
                   session_len=(1, 64), nv_grid=SERVE_NV_GRID, p_program: float = 0.5):
    """The request stream of the serving workload without its data: open-loop
    Poisson arrivals at ``rate`` req/s (exponential gaps); sessions of
    session_len requests (uniform) whose variable count is drawn uniformly from
    nv_grid; requests of all sessions interleaved at random; each request a
    program (p_program) or a trace of floor(2^U(a, b)) ops.  Returns a dict of
    numpy arrays: arrival (s), session, nv, kind (0 trace / 1 program), n_ops
    (traces), offset (a uniform start in [0, 2^24 - n_ops], for slicing an op
    pool), prog_index (programs: the generator index)."""
    rng = np.random.default_rng(seed)
    t = np.cumsum(rng.exponential(1.0 / rate, n_requests))
    lens, nvs = [], []
    while sum(lens) < n_requests:
        lens.append(min(int(rng.integers(session_len[0], session_len[1] + 1)), n_requests - sum(lens)))
        nvs.append(int(rng.choice(nv_grid)))
    order = np.repeat(np.arange(len(lens)), lens)
    rng.shuffle(order)
    kind = (rng.random(n_requests) < p_program).astype(np.int32)
    n_ops = np.floor(2.0 ** rng.uniform(trace_log2[0], trace_log2[1], n_requests)).astype(np.int64)
    offset = (rng.random(n_requests) * ((1 << 24) - n_ops + 1)).astype(np.int64)
    prog_index = np.cumsum(kind) - 1
    return dict(arrival=t, session=order.astype(np.int64), nv=np.array(nvs, np.int32)[order], kind=kind,
                n_ops=np.where(kind == 0, n_ops, 0), offset=np.where(kind == 0, offset, 0),
                prog_index=np.where(kind == 1, prog_index, -1))


def serve_requests(rate: float, n_requests: int = 10_000, seed: int = 4,
                   trace_log2=(10.0, 24.0), session_len=(1, 64), vars_range=(64, 4096),
                   p_program: float = 0.5, **prog_kw):
    """Open-loop Poisson arrivals (exponential gaps at ``rate`` req/s).
    Sessions of session_len requests (uniform) over vars_range vars (uniform);
    a session's requests arrive in order.  Each request is a program drawn from
    the program distribution or a trace of floor(2^U(a, b)) ops with the Zipf
    trace's kind mix and a uniform var over the session's vars.  Returns a list
    of request dicts sorted by arrival time (seconds)."""
    rng = np.random.default_rng(seed)
    t = np.cumsum(rng.exponential(1.0 / rate, n_requests))
    sessions = []
    sid = 0
    assigned = 0
    while assigned < n_requests:
        k = int(rng.integers(session_len[0], session_len[1] + 1))
        k = min(k, n_requests - assigned)
        sessions.append((sid, k, int(rng.integers(vars_range[0], vars_range[1] + 1))))
        assigned += k
        sid += 1
    # interleave sessions: each arrival slot picks a random session with requests left
    order = np.repeat(np.arange(len(sessions)), [s[1] for s in sessions])
    rng.shuffle(order)
    reqs = []
    prog_index = 0
    for i, s in enumerate(order):
        sid, _, nv = sessions[s]
        if rng.random() < p_program:
            kw = dict(prog_kw)
            kw.update(vars_lo=nv, vars_hi=nv)
            pr = programs(1, seed=seed * 1_000_003 + 7, first=prog_index, **kw)
            prog_index += 1
            reqs.append(dict(arrival=float(t[i]), session=int(sid), n_vars=nv, kind="program",
                             tok=pr["tok"], payload=pr["payload"]))
        else:
            n = int(math.floor(2.0 ** rng.uniform(*trace_log2)))
            kind = rng.choice(5, size=n, p=KIND_MIX)
            side = rng.integers(0, 2, n)
            var = rng.integers(0, nv, n)
            reqs.append(dict(arrival=float(t[i]), session=int(sid), n_vars=nv, kind="trace",
                             kind_side=(kind | (side << 4)).astype(np.uint8),
                             var=var.astype(np.int32)))
    return reqs
