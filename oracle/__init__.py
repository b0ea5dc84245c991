"""Plain CPU oracle for GP population evaluation -- TEST INFRASTRUCTURE ONLY.

Only ``tests/``, ``__graft_entry__.smoke()`` and ``bench.py``'s CPU-baseline leg
(and its ``--impl reference`` arm) may import this package.  It shares no code with the
CUDA library in ``paper_1601_00221_gb300`` and the CUDA library never calls it.

The C sources (``oracle.c``: {+,-,*,/} trees, Boolean trees, register
programs; ``oracle_fset.c``: the full float function sets of Sec. 4.2, the
fitness measures, per-case output enclosures) evaluate every fitness case
separately, node by node, exactly as the tree defines it (Chitty, Sec. 3-4:
the two-dimensional stack changes the schedule, not the values).  This module
builds them with gcc (``-O2 -ffp-contract=off``, no fast-math) and wraps them
with ctypes.

Parity unpinned: none -- every function here is pinned by ``tests/test_oracle_pins.py``
and ``tests/test_oracle_fset.py`` (closed forms, brute-force truth tables,
numpy binary32 arithmetic, exact sums, sampled admissible implementations).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRCS = [os.path.join(_HERE, "oracle.c"), os.path.join(_HERE, "oracle_fset.c")]
_HDR = os.path.join(_HERE, "oracle.h")
_BUILD = os.path.join(_HERE, "_build")
_SO = os.path.join(_BUILD, "liboracle.so")
CFLAGS = ["-O2", "-std=c11", "-ffp-contract=off", "-fno-fast-math", "-fPIC", "-shared",
          "-Wall", "-Wextra", "-Wno-unused-parameter"]

# opcodes of the user token format (same numbers as the public header; defined
# here independently because the oracle shares no code with the library)
ADD, SUB, MUL, DIV, VAR, CONST, AND, OR, NAND, NOR, IF = range(1, 12)
SIN, COS, EXP, LOG, GT, LT, EQ = range(12, 19)
# fitness measures
FIT_ABS, FIT_MSE, FIT_CLASS = 0, 1, 2

_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile the C sources into oracle/_build/liboracle.so (no-op when up to date)."""
    os.makedirs(_BUILD, exist_ok=True)
    newest = max(os.path.getmtime(f) for f in _SRCS + [_HDR])
    if force or not os.path.exists(_SO) or os.path.getmtime(_SO) < newest:
        tmp = _SO + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", *CFLAGS, "-o", tmp, *_SRCS, "-lm"])
        os.replace(tmp, _SO)
    return _SO


def lib() -> ctypes.CDLL:
    global _lib
    with _lock:
        if _lib is None:
            build()
            L = ctypes.CDLL(_SO)
            P = ctypes.c_void_p
            i32, i64 = ctypes.c_int32, ctypes.c_int64
            L.oracle_apply_op.argtypes = [ctypes.c_int, ctypes.c_float, ctypes.c_float]
            L.oracle_apply_op.restype = ctypes.c_float
            for name in ("oracle_tree_outputs", "oracle_tree_outputs_stack"):
                getattr(L, name).argtypes = [P, i64, P, i32, i64, P]
                getattr(L, name).restype = ctypes.c_int
            L.oracle_tree_nodes.argtypes = [P, i64]
            L.oracle_tree_nodes.restype = i64
            L.oracle_tree_fitness.argtypes = [P, i64, P, i32, i64, P, P]
            L.oracle_tree_fitness.restype = ctypes.c_int
            L.oracle_population_fitness.argtypes = [P, P, P, i32, i32, P, i32, i64, P, P]
            L.oracle_population_fitness.restype = ctypes.c_int
            L.oracle_bool_outputs.argtypes = [P, i64, P, i32, i64, P]
            L.oracle_bool_outputs.restype = ctypes.c_int
            L.oracle_bool_hits.argtypes = [P, i64, P, i32, i64, P, P]
            L.oracle_bool_hits.restype = ctypes.c_int
            L.oracle_bool_population_hits.argtypes = [P, P, P, i32, i32, P, i32, i64, P, P]
            L.oracle_bool_population_hits.restype = ctypes.c_int
            L.oracle_linear_outputs.argtypes = [P, P, P, P, i32, P, i32, i64, P]
            L.oracle_linear_outputs.restype = ctypes.c_int
            L.oracle_linear_population_fitness.argtypes = [P, P, P, i32, i32, P, i32, i64, P, P]
            L.oracle_linear_population_fitness.restype = ctypes.c_int
            L.oracle_fset_arity.argtypes = [ctypes.c_int]
            L.oracle_fset_arity.restype = ctypes.c_int
            L.oracle_fset_outputs.argtypes = [P, i64, P, i32, i64, P]
            L.oracle_fset_outputs.restype = ctypes.c_int
            L.oracle_fset_enclosure.argtypes = [P, i64, P, i32, i64, P, P, P]
            L.oracle_fset_enclosure.restype = ctypes.c_int
            L.oracle_fitness_of_outputs.argtypes = [P, P, i64, i32, P]
            L.oracle_fitness_of_outputs.restype = ctypes.c_int
            L.oracle_fitness_enclosure.argtypes = [P, P, P, P, i64, i32, P, P, P, P]
            L.oracle_fitness_enclosure.restype = ctypes.c_int
            L.oracle_fset_population_fitness.argtypes = [P, P, P, i32, i32, P, i32, i64, P, i32, P]
            L.oracle_fset_population_fitness.restype = ctypes.c_int
            _lib = L
    return _lib


class OracleError(RuntimeError):
    pass


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p)


def _c(a, dtype):
    return np.ascontiguousarray(a, dtype=dtype)


def _check(rc: int, what: str):
    if rc != 0:
        raise OracleError(f"{what}: oracle error code {rc}")


def apply_op(op: int, a: float, b: float) -> np.float32:
    return np.float32(lib().oracle_apply_op(op, np.float32(a), np.float32(b)))


def tree_nodes(prog) -> int:
    p = _c(prog, np.uint32)
    n = lib().oracle_tree_nodes(_ptr(p), p.size)
    if n < 0:
        raise OracleError(f"tree_nodes: error {n}")
    return int(n)


def tree_outputs(prog, cases, method: str = "recursive") -> np.ndarray:
    """Per-case binary32 outputs of one prefix tree; cases is [n_inputs, n_cases]."""
    p = _c(prog, np.uint32)
    x = _c(cases, np.float32)
    if x.ndim == 1:
        x = x[None, :]
    n_inputs, n_cases = x.shape
    out = np.empty(n_cases, np.float32)
    fn = lib().oracle_tree_outputs if method == "recursive" else lib().oracle_tree_outputs_stack
    _check(fn(_ptr(p), p.size, _ptr(x), n_inputs, n_cases, _ptr(out)), "tree_outputs")
    return out


def tree_fitness(prog, cases, targets) -> float:
    p = _c(prog, np.uint32)
    x = _c(cases, np.float32)
    if x.ndim == 1:
        x = x[None, :]
    y = _c(targets, np.float32)
    f = np.zeros(1, np.float64)
    _check(lib().oracle_tree_fitness(_ptr(p), p.size, _ptr(x), x.shape[0], x.shape[1],
                                     _ptr(y), _ptr(f)), "tree_fitness")
    return float(f[0])


def population_fitness(programs, offsets, lengths, cases, targets, p_range=None) -> np.ndarray:
    """Fitness of programs [p_begin, p_end) (all by default); others left NaN."""
    w = _c(programs, np.uint32)
    off = _c(offsets, np.int64)
    ln = _c(lengths, np.int32)
    x = _c(cases, np.float32)
    if x.ndim == 1:
        x = x[None, :]
    y = _c(targets, np.float32)
    n = ln.size
    b, e = (0, n) if p_range is None else p_range
    out = np.full(n, np.nan, np.float64)
    _check(lib().oracle_population_fitness(_ptr(w), _ptr(off), _ptr(ln), b, e, _ptr(x),
                                           x.shape[0], x.shape[1], _ptr(y), _ptr(out)),
           "population_fitness")
    return out


def bool_outputs(prog, case_bits) -> np.ndarray:
    p = _c(prog, np.uint32)
    cb = _c(case_bits, np.uint32)
    if cb.ndim == 1:
        cb = cb[None, :]
    n_inputs, n_words = cb.shape
    out = np.empty(n_words, np.uint32)
    _check(lib().oracle_bool_outputs(_ptr(p), p.size, _ptr(cb), n_inputs, n_words, _ptr(out)),
           "bool_outputs")
    return out


def bool_hits(prog, case_bits, n_cases, target_bits) -> int:
    p = _c(prog, np.uint32)
    cb = _c(case_bits, np.uint32)
    if cb.ndim == 1:
        cb = cb[None, :]
    t = _c(target_bits, np.uint32)
    h = np.zeros(1, np.uint64)
    _check(lib().oracle_bool_hits(_ptr(p), p.size, _ptr(cb), cb.shape[0], n_cases, _ptr(t),
                                  _ptr(h)), "bool_hits")
    return int(h[0])


def bool_population_hits(programs, offsets, lengths, case_bits, n_cases, target_bits,
                         p_range=None) -> np.ndarray:
    w = _c(programs, np.uint32)
    off = _c(offsets, np.int64)
    ln = _c(lengths, np.int32)
    cb = _c(case_bits, np.uint32)
    t = _c(target_bits, np.uint32)
    n = ln.size
    b, e = (0, n) if p_range is None else p_range
    out = np.zeros(n, np.uint64)
    _check(lib().oracle_bool_population_hits(_ptr(w), _ptr(off), _ptr(ln), b, e, _ptr(cb),
                                             cb.shape[0], n_cases, _ptr(t), _ptr(out)),
           "bool_population_hits")
    return out


def linear_outputs(instr, cases) -> np.ndarray:
    """instr: uint8 [n_instr, 4] rows (dst, op, a, b); cases: [n_inputs, n_cases]."""
    ins = _c(instr, np.uint8).reshape(-1, 4)
    d, o, a, b = (np.ascontiguousarray(ins[:, i]) for i in range(4))
    x = _c(cases, np.float32)
    if x.ndim == 1:
        x = x[None, :]
    out = np.empty(x.shape[1], np.float32)
    _check(lib().oracle_linear_outputs(_ptr(d), _ptr(o), _ptr(a), _ptr(b), ins.shape[0],
                                       _ptr(x), x.shape[0], x.shape[1], _ptr(out)),
           "linear_outputs")
    return out


def linear_population_fitness(instr, offsets, lengths, cases, targets, p_range=None) -> np.ndarray:
    ins = _c(instr, np.uint8).reshape(-1)
    off = _c(offsets, np.int64)
    ln = _c(lengths, np.int32)
    x = _c(cases, np.float32)
    y = _c(targets, np.float32)
    n = ln.size
    b, e = (0, n) if p_range is None else p_range
    out = np.full(n, np.nan, np.float64)
    _check(lib().oracle_linear_population_fitness(_ptr(ins), _ptr(off), _ptr(ln), b, e,
                                                  _ptr(x), x.shape[0], x.shape[1], _ptr(y),
                                                  _ptr(out)), "linear_population_fitness")
    return out


# ---------------------------------------------------------------------------
# full float function sets (oracle_fset.c)
# ---------------------------------------------------------------------------
def _cases2d(cases):
    x = _c(cases, np.float32)
    return x[None, :] if x.ndim == 1 else x


def fset_arity(op: int) -> int:
    return int(lib().oracle_fset_arity(op))


def fset_outputs(prog, cases) -> np.ndarray:
    """Per-case outputs of a tree over the full function sets (transcendental
    nodes: the binary32 value nearest the binary64 libm result)."""
    p = _c(prog, np.uint32)
    x = _cases2d(cases)
    out = np.empty(x.shape[1], np.float32)
    _check(lib().oracle_fset_outputs(_ptr(p), p.size, _ptr(x), x.shape[0], x.shape[1], _ptr(out)),
           "fset_outputs")
    return out


def fset_enclosure(prog, cases):
    """(lo, hi, may_nan): every admissible evaluation of case c is in
    [lo[c], hi[c]] or NaN where may_nan[c]; lo > hi means NaN only."""
    p = _c(prog, np.uint32)
    x = _cases2d(cases)
    n = x.shape[1]
    lo = np.empty(n, np.float32)
    hi = np.empty(n, np.float32)
    nan = np.empty(n, np.uint8)
    _check(lib().oracle_fset_enclosure(_ptr(p), p.size, _ptr(x), x.shape[0], n, _ptr(lo), _ptr(hi),
                                       _ptr(nan)), "fset_enclosure")
    return lo, hi, nan.astype(bool)


def fitness_of_outputs(out, targets, kind: int) -> float:
    o = _c(out, np.float32)
    y = _c(targets, np.float32)
    f = np.zeros(1, np.float64)
    _check(lib().oracle_fitness_of_outputs(_ptr(o), _ptr(y), o.size, kind, _ptr(f)),
           "fitness_of_outputs")
    return float(f[0])


def fitness_enclosure(lo, hi, may_nan, targets, kind: int):
    """(f_lo, f_hi, may_inf, must_inf) of a program from its case enclosures."""
    lo = _c(lo, np.float32)
    hi = _c(hi, np.float32)
    nan = _c(may_nan, np.uint8)
    y = _c(targets, np.float32)
    r = np.zeros(2, np.float64)
    flags = np.zeros(2, np.int32)
    _check(lib().oracle_fitness_enclosure(_ptr(lo), _ptr(hi), _ptr(nan), _ptr(y), lo.size, kind,
                                          _ptr(r[0:]), ctypes.c_void_p(r.ctypes.data + 8),
                                          _ptr(flags[0:]), ctypes.c_void_p(flags.ctypes.data + 4)),
           "fitness_enclosure")
    return float(r[0]), float(r[1]), bool(flags[0]), bool(flags[1])


def fset_population_fitness(programs, offsets, lengths, cases, targets, kind: int = FIT_ABS,
                            p_range=None) -> np.ndarray:
    w = _c(programs, np.uint32)
    off = _c(offsets, np.int64)
    ln = _c(lengths, np.int32)
    x = _cases2d(cases)
    y = _c(targets, np.float32)
    n = ln.size
    b, e = (0, n) if p_range is None else p_range
    out = np.full(n, np.nan, np.float64)
    _check(lib().oracle_fset_population_fitness(_ptr(w), _ptr(off), _ptr(ln), b, e, _ptr(x),
                                                x.shape[0], x.shape[1], _ptr(y), kind, _ptr(out)),
           "fset_population_fitness")
    return out
