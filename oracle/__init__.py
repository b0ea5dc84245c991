"""Plain CPU oracle for GP population evaluation -- TEST INFRASTRUCTURE ONLY.

Only ``tests/``, ``__graft_entry__.smoke()`` and ``bench.py``'s CPU-baseline leg
(and its ``--impl reference`` arm) may import this package.  It shares no code with the
CUDA library in ``paper_1601_00221_gb300`` and the CUDA library never calls it.

The C source (``oracle.c``) evaluates every fitness case separately, node by
node, exactly as the tree defines it (Chitty, Sec. 3-4: the two-dimensional
stack changes the schedule, not the values).  This module builds it with gcc
(``-O2 -ffp-contract=off``, no fast-math) and wraps it with ctypes.

Parity unpinned: none -- every function here is pinned by ``tests/test_oracle_pins.py``
(closed forms, brute-force truth tables, numpy binary32 arithmetic, exact sums).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_HDR = os.path.join(_HERE, "oracle.h")
_BUILD = os.path.join(_HERE, "_build")
_SO = os.path.join(_BUILD, "liboracle.so")
CFLAGS = ["-O2", "-std=c11", "-ffp-contract=off", "-fno-fast-math", "-fPIC", "-shared",
          "-Wall", "-Wextra", "-Wno-unused-parameter"]

# opcodes of the user token format (same numbers as the public header; defined
# here independently because the oracle shares no code with the library)
ADD, SUB, MUL, DIV, VAR, CONST, AND, OR, NAND, NOR, IF = range(1, 12)

_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile oracle.c into oracle/_build/liboracle.so (no-op when up to date)."""
    os.makedirs(_BUILD, exist_ok=True)
    newest = max(os.path.getmtime(_SRC), os.path.getmtime(_HDR))
    if force or not os.path.exists(_SO) or os.path.getmtime(_SO) < newest:
        tmp = _SO + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", *CFLAGS, "-o", tmp, _SRC, "-lm"])
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
