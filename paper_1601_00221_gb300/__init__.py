"""Python binding of libgpeval.so, the GB300 (sm_103a) GP population evaluator.

The binding only marshals arguments: every step of an evaluation runs in the
library's CUDA kernels (``csrc/``), and the host encoder runs in the library's
C++ code.  PyTorch supplies device memory and streams.  There is no fallback:
if the library is missing or fails to load, importing the evaluation entry
points raises.

Function names follow ``include/gpeval.h``.
"""
from __future__ import annotations

import ctypes
import os
from dataclasses import dataclass
from typing import Optional

import numpy as np

from . import build as _build

__all__ = [
    "GPError", "lib", "Config", "EncodedPopulation",
    "encode_tree", "encode_population", "encode_linear_population",
    "eval_population", "eval_outputs", "eval_population_bool",
    "set_config", "reset_config", "get_config", "last_error", "shutdown", "version", "Server", "RUN_FLOAT", "RUN_BOOL",
    "eval_population_noalloc", "eval_segments", "eval_population_split", "MAX_SEGMENTS", "autotune_population", "autotune_population_ex",
    "autotune_population_bool", "autotune_save", "autotune_load", "autotune_clear", "eval_launches",
    "autotune_split_record",
    "KIND_SFORM", "KIND_RPN", "KIND_LINEAR", "KIND_BOOL", "KIND_SFORM_EXT", "KIND_RPN_EXT",
    "ORDER_PAPER",
    "ORDER_MIN_DEPTH", "VARIANT_AUTO", "VARIANT_REGISTER", "VARIANT_LOCAL", "VARIANT_LANES",
    "VARIANT_EXTENDED", "VARIANT_EXTENDED_RPN", "VARIANT_REGISTER_FILE", "VARIANT_WARPS", "FITNESS_SUM_ABS", "FITNESS_MSE", "FITNESS_CLASS",
    "encode_population_device", "EvolveParams", "Evolver",
]

KIND_SFORM, KIND_RPN, KIND_LINEAR, KIND_BOOL, KIND_SFORM_EXT, KIND_RPN_EXT = 1, 2, 3, 4, 5, 6
ORDER_PAPER, ORDER_MIN_DEPTH = 0, 1
VARIANT_AUTO, VARIANT_REGISTER, VARIANT_LOCAL, VARIANT_LANES, VARIANT_EXTENDED = 0, 1, 2, 3, 4
VARIANT_EXTENDED_RPN = 5
VARIANT_REGISTER_FILE = 6
VARIANT_WARPS = 7
FITNESS_SUM_ABS, FITNESS_MSE, FITNESS_CLASS = 0, 1, 2
STACK_LEVELS = 8
MAX_INSTR = 1024

_STATUS = {0: "GP_OK", 1: "GP_ERR_INVALID_ARG", 2: "GP_ERR_PROGRAM", 3: "GP_ERR_CUDA",
           4: "GP_ERR_OOM", 5: "GP_ERR_TIMEOUT", 6: "GP_ERR_NOT_IMPLEMENTED", 7: "GP_ERR_BUSY",
           8: "GP_ERR_CANCELLED"}
RUN_FLOAT, RUN_BOOL = 1, 2


class GPError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"{_STATUS.get(code, code)}: {msg}")
        self.code = code


class _ProgInfo(ctypes.Structure):
    _fields_ = [("n_nodes", ctypes.c_int32), ("n_instr", ctypes.c_int32),
                ("max_depth", ctypes.c_int32), ("stack_reads", ctypes.c_int32),
                ("max_input", ctypes.c_int32), ("words", ctypes.c_int32),
                ("extended", ctypes.c_int32), ("inputs_used", ctypes.c_int32)]


class _ServerOpts(ctypes.Structure):
    _fields_ = [("n_streams", ctypes.c_int32), ("max_inflight", ctypes.c_int32),
                ("max_queued", ctypes.c_int32), ("max_merge", ctypes.c_int32),
                ("memory_budget", ctypes.c_int64), ("variant", ctypes.c_int32),
                ("k", ctypes.c_int32), ("block", ctypes.c_int32), ("chunk_cases", ctypes.c_int32),
                ("fitness", ctypes.c_int32), ("tile_inputs", ctypes.c_int32),
                ("stack_registers", ctypes.c_int32), ("max_instructions", ctypes.c_int32)]


class RequestInfo(ctypes.Structure):
    _fields_ = [("status", ctypes.c_int32), ("n_progs", ctypes.c_int32), ("gpop", ctypes.c_int64),
                ("t_submit_us", ctypes.c_double), ("t_admit_us", ctypes.c_double),
                ("t_done_us", ctypes.c_double)]


class ServerStats(ctypes.Structure):
    _fields_ = [("submitted", ctypes.c_int64), ("completed", ctypes.c_int64),
                ("failed", ctypes.c_int64), ("cancelled", ctypes.c_int64),
                ("launches", ctypes.c_int64), ("gpop_completed", ctypes.c_int64),
                ("p50_latency_us", ctypes.c_double), ("p99_latency_us", ctypes.c_double),
                ("max_latency_us", ctypes.c_double), ("busy_s", ctypes.c_double),
                ("gpop_per_s", ctypes.c_double)]

    def as_dict(self):
        return {f: getattr(self, f) for f, _ in self._fields_}


class Config(ctypes.Structure):
    """gp_config: variant, k (cases per thread per pass), block, chunk_cases
    (0 = choose), fitness (FITNESS_SUM_ABS, FITNESS_MSE or FITNESS_CLASS),
    tile_inputs (inputs per case the shared-memory tile holds, 0 = all),
    stack_registers, max_instructions (the longest program's instructions,
    0 = the API maximum: the per-block program buffer)."""
    _fields_ = [("variant", ctypes.c_int32), ("k", ctypes.c_int32), ("block", ctypes.c_int32),
                ("chunk_cases", ctypes.c_int32), ("fitness", ctypes.c_int32),
                ("tile_inputs", ctypes.c_int32), ("stack_registers", ctypes.c_int32),
                ("max_instructions", ctypes.c_int32)]

    def __repr__(self):
        return (f"Config(variant={self.variant}, k={self.k}, block={self.block}, "
                f"chunk_cases={self.chunk_cases}, fitness={self.fitness}, "
                f"tile_inputs={self.tile_inputs}, stack_registers={self.stack_registers}, "
                f"max_instructions={self.max_instructions})")


_lib = None


def lib(rebuild: bool = False) -> ctypes.CDLL:
    """Loads (building first if needed) libgpeval.so.  Raises if it cannot."""
    global _lib
    if _lib is not None and not rebuild:
        return _lib
    path = _build.LIB
    if rebuild or not os.path.exists(path):
        path = _build.build()
    L = ctypes.CDLL(path)
    P, i32, i64 = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64
    sig = {
        "gp_encode_tree": [P, i64, i32, i32, P, i64, P],
        "gp_encode_population": [P, P, P, i32, i32, i32, P, i64, P, P, P, P, P, P],
        "gp_encode_linear_population": [P, P, P, i32, P, i64, P, P, P, P, P],
        "gp_eval_population": [P, P, P, i32, P, i32, i64, P, P, P],
        "gp_eval_population_ex": [P, P, P, i32, P, i32, i64, P, P, P, P, P],
        "gp_eval_outputs": [P, P, P, i32, P, i32, i64, P, P, P],
        "gp_eval_population_bool": [P, P, P, i32, P, i32, i64, P, P, P],
        "gp_eval_population_bool_ex": [P, P, P, i32, P, i32, i64, P, P, P, P, P],
        "gp_set_config": [P],
        "gp_get_config": [P],
        "gp_last_error": [P, P],
        "gp_shutdown": [],
        "gp_eval_population_noalloc": [P, P, P, i32, P, i32, i64, P, P, P],
        "gp_eval_segments": [P, P, P, P, i32, i32, P, P],
        "gp_eval_population_split": [P, P, P, i32, P, i32, i64, P, P, i32, P, P, P],
        "gp_server_create": [P, P],
        "gp_server_register_run": [P, i32, P, i32, i64, P, P],
        "gp_server_submit": [P, i32, P, P, P, i32, i64, P, P],
        "gp_server_poll": [P, ctypes.c_uint64, P],
        "gp_server_wait": [P, ctypes.c_uint64, i64, P],
        "gp_server_cancel": [P, ctypes.c_uint64],
        "gp_server_get_stats": [P, P],
        "gp_server_destroy": [P],
        "gp_autotune_population": [P, P, P, i32, P, i32, i64, P, i32, P, P],
        "gp_autotune_clear": [],
        "gp_autotune_population_ex": [P, P, P, i32, P, i32, i64, P, P, i32, P, P],
        "gp_autotune_population_bool": [P, P, P, i32, P, i32, i64, P, P, i32, P, P],
        "gp_autotune_save": [ctypes.c_char_p],
        "gp_autotune_load": [ctypes.c_char_p],
        "gp_autotune_split_record": [i32, i32, i64, i32, P, P, P],
        "gp_eval_launches": [i32, i64, P],
        "gp_encode_population_device": [P, P, P, i32, i32, P, P, P, P],
        "gp_encode_slots_device": [P, i32, P, P],
        "gp_evolve_create": [P, P, P, P, P, i32, i64, P, P],
        "gp_evolve_run": [P, i32],
        "gp_evolve_read": [P, P, P, P, P, P],
        "gp_evolve_destroy": [P],
    }
    for name, args in sig.items():
        fn = getattr(L, name)
        fn.argtypes = args
        fn.restype = ctypes.c_int
    L.gp_error_string.argtypes = []
    L.gp_error_string.restype = ctypes.c_char_p
    L.gp_version.argtypes = []
    L.gp_version.restype = ctypes.c_int32
    _lib = L
    return L


def _check(rc: int):
    if rc != 0:
        raise GPError(rc, lib().gp_error_string().decode(errors="replace"))


def _np_ptr(a: Optional[np.ndarray]):
    return None if a is None else a.ctypes.data_as(ctypes.c_void_p)


def version() -> int:
    return int(lib().gp_version())


# ---------------------------------------------------------------------------
# host encoder
# ---------------------------------------------------------------------------
@dataclass
class EncodedPopulation:
    words: np.ndarray      # uint32, 16-byte aligned programs back to back
    offsets: np.ndarray    # int64 word offsets
    lengths: np.ndarray    # int32 word lengths
    nodes: int             # total tree nodes (GPop unit per case)
    kind: int
    order: int
    info: Optional[np.ndarray] = None  # structured per-program info (tree kinds)

    @property
    def n(self) -> int:
        return int(self.lengths.size)

    @property
    def extended(self) -> bool:
        """Some program uses the extended float functions (needs VARIANT_EXTENDED)."""
        if self.kind not in (KIND_SFORM, KIND_RPN) or self.n == 0:
            return False
        kinds = self.words[self.offsets] & 0xFF
        return bool(np.any((kinds == KIND_SFORM_EXT) | (kinds == KIND_RPN_EXT)))

    @property
    def max_inputs_used(self) -> int:
        """The most distinct inputs any tree reads (0 if unknown or none)."""
        if self.info is None or self.n == 0 or "inputs_used" not in self.info.dtype.names:
            return 0
        return int(self.info["inputs_used"].max())

    @property
    def max_instructions(self) -> int:
        """Instructions of the longest program (0 for an empty population: the
        API maximum); an encoded program of n instructions takes 4 + 4 n words."""
        if self.n == 0:
            return 0
        if self.info is not None and "n_instr" in self.info.dtype.names:
            return max(int(self.info["n_instr"].max()), 1)
        return max((int(self.lengths.max()) - 4) // 4, 1)

    def config(self, fitness: int = FITNESS_SUM_ABS, k: int = 0, block: int = 0,
               chunk_cases: int = 0) -> "Config":
        """A configuration that can run this population with the given fitness
        measure: the extended interpreter when some program needs it, and a
        staged-input tile and a program buffer no larger than the population
        needs."""
        variant = VARIANT_AUTO
        if self.extended:
            variant = VARIANT_EXTENDED_RPN if self.kind == KIND_RPN else VARIANT_EXTENDED
        elif self.kind == KIND_LINEAR:
            variant = VARIANT_REGISTER_FILE
        tile = max(self.max_inputs_used, 1) if self.kind in (KIND_SFORM, KIND_RPN) else 0
        return Config(variant, k, block, chunk_cases, fitness, tile, 0, self.max_instructions)

    def to_device(self, device="cuda"):
        import torch
        return (torch.from_numpy(self.words.view(np.int32)).to(device),
                torch.from_numpy(self.offsets).to(device),
                torch.from_numpy(self.lengths).to(device))


def encode_tree(prefix, kind: int = KIND_SFORM, order: int = ORDER_MIN_DEPTH):
    """One prefix tree -> (encoded uint32 words, info dict)."""
    p = np.ascontiguousarray(prefix, dtype=np.uint32)
    info = _ProgInfo()
    cap = 4 + 4 * max(1, p.size)
    out = np.zeros(cap, np.uint32)
    _check(lib().gp_encode_tree(_np_ptr(p), p.size, kind, order, _np_ptr(out), cap,
                                ctypes.byref(info)))
    d = {f: getattr(info, f) for f, _ in _ProgInfo._fields_}
    return out[:info.words].copy(), d


def encode_population(words, offsets, lengths, kind: int = KIND_SFORM,
                      order: int = ORDER_MIN_DEPTH, with_info: bool = False,
                      out: Optional[np.ndarray] = None) -> EncodedPopulation:
    """Encodes a population in one call (the output is sized by the bound of
    4 + 4 * lengths[p] words per program).  `out` (uint32, 16-byte aligned)
    may supply the buffer, e.g. a pinned host array reused across calls.
    The per-program info is always kept (`with_info` is accepted for older
    callers)."""
    w = np.ascontiguousarray(words, np.uint32)
    off = np.ascontiguousarray(offsets, np.int64)
    ln = np.ascontiguousarray(lengths, np.int32)
    n = int(ln.size)
    cap = int(4 * n + 4 * int(ln.sum())) if n else 4
    if out is None or out.size < cap:
        out = _aligned_empty(max(cap, 4))
    total = ctypes.c_int64(0)
    nodes = ctypes.c_int64(0)
    bad = ctypes.c_int32(-1)
    out_off = np.zeros(n, np.int64)
    out_len = np.zeros(n, np.int32)
    info = (_ProgInfo * n)()
    _check(lib().gp_encode_population(_np_ptr(w), _np_ptr(off), _np_ptr(ln), n, kind, order,
                                      _np_ptr(out), out.size, _np_ptr(out_off), _np_ptr(out_len),
                                      ctypes.byref(total), ctypes.byref(nodes),
                                      ctypes.cast(info, ctypes.c_void_p),
                                      ctypes.byref(bad)))
    arr = np.ctypeslib.as_array(info).copy() if n else None
    return EncodedPopulation(out[:max(int(total.value), 4)], out_off, out_len, int(nodes.value),
                             kind, order, arr)


def encode_linear_population(instr, offsets, lengths) -> EncodedPopulation:
    ins = np.ascontiguousarray(instr, np.uint8).reshape(-1)
    off = np.ascontiguousarray(offsets, np.int64)
    ln = np.ascontiguousarray(lengths, np.int32)
    n = int(ln.size)
    total = ctypes.c_int64(0)
    nodes = ctypes.c_int64(0)
    bad = ctypes.c_int32(-1)
    L = lib()
    _check(L.gp_encode_linear_population(_np_ptr(ins), _np_ptr(off), _np_ptr(ln), n, None, 0,
                                         None, None, ctypes.byref(total), ctypes.byref(nodes),
                                         ctypes.byref(bad)))
    out = _aligned_empty(max(int(total.value), 4))
    out_off = np.zeros(n, np.int64)
    out_len = np.zeros(n, np.int32)
    _check(L.gp_encode_linear_population(_np_ptr(ins), _np_ptr(off), _np_ptr(ln), n,
                                         _np_ptr(out), out.size, _np_ptr(out_off),
                                         _np_ptr(out_len), ctypes.byref(total),
                                         ctypes.byref(nodes), ctypes.byref(bad)))
    return EncodedPopulation(out, out_off, out_len, int(nodes.value), KIND_LINEAR, 0)


def _aligned_empty(n_words: int) -> np.ndarray:
    buf = np.zeros(n_words + 4, np.uint32)
    shift = (-(buf.ctypes.data // 4)) % 4
    return buf[shift:shift + n_words]


# ---------------------------------------------------------------------------
# evaluation (torch tensors on the current CUDA device)
# ---------------------------------------------------------------------------
def _tptr(t):
    return None if t is None else ctypes.c_void_p(t.data_ptr())


def _stream(stream):
    import torch
    s = stream if stream is not None else torch.cuda.current_stream()
    return ctypes.c_void_p(s.cuda_stream)


def _cfg(config):
    if config is None:
        return None
    if isinstance(config, Config):
        return ctypes.byref(config)
    c = Config(**config)
    return ctypes.byref(c)


def eval_population(programs, offsets, lengths, cases, targets, fitness_out=None, outputs=None,
                    config=None, stream=None):
    """Fitness (float64 [n]) of encoded float programs (GP_KIND_SFORM/RPN/LINEAR).

    programs int32/uint32 words, offsets int64, lengths int32, cases float32
    [n_inputs, n_cases], targets float32 [n_cases]; all CUDA tensors.
    Returns fitness_out (allocated when None).  `outputs` (float32
    [n, n_cases]) optionally receives per-case outputs.
    """
    import torch
    n = int(lengths.numel())
    n_inputs, n_cases = (int(cases.shape[0]), int(cases.shape[1])) if cases.dim() == 2 else (1, int(cases.numel()))
    if fitness_out is None:
        fitness_out = torch.empty(n, dtype=torch.float64, device=cases.device)
    _check(lib().gp_eval_population_ex(_tptr(programs), _tptr(offsets), _tptr(lengths), n,
                                       _tptr(cases), n_inputs, n_cases, _tptr(targets),
                                       _tptr(fitness_out), _tptr(outputs), _cfg(config),
                                       _stream(stream)))
    return fitness_out


def eval_population_split(programs, offsets, lengths, cases, targets, split_inputs, narrow, wide,
                          fitness_out=None, stream=None):
    """gp_eval_population_split: programs reading at most split_inputs
    distinct inputs under `narrow`, the others under `wide` (Configs)."""
    import torch
    n = int(lengths.numel())
    n_inputs, n_cases = (int(cases.shape[0]), int(cases.shape[1])) if cases.dim() == 2 else (1, int(cases.numel()))
    if fitness_out is None:
        fitness_out = torch.empty(n, dtype=torch.float64, device=cases.device)
    _check(lib().gp_eval_population_split(_tptr(programs), _tptr(offsets), _tptr(lengths), n, _tptr(cases),
                                          n_inputs, n_cases, _tptr(targets), _tptr(fitness_out), int(split_inputs),
                                          _cfg(narrow), _cfg(wide), _stream(stream)))
    return fitness_out


def eval_outputs(programs, offsets, lengths, cases, outputs=None, config=None, stream=None):
    import torch
    n = int(lengths.numel())
    n_inputs, n_cases = (int(cases.shape[0]), int(cases.shape[1])) if cases.dim() == 2 else (1, int(cases.numel()))
    if outputs is None:
        outputs = torch.empty((n, n_cases), dtype=torch.float32, device=cases.device)
    _check(lib().gp_eval_outputs(_tptr(programs), _tptr(offsets), _tptr(lengths), n,
                                 _tptr(cases), n_inputs, n_cases, _tptr(outputs), _cfg(config),
                                 _stream(stream)))
    return outputs


def eval_population_bool(programs, offsets, lengths, case_bits, n_cases, target_bits,
                         hits_out=None, out_words=None, config=None, stream=None):
    """Hit counts (int64 tensor [n], exact) of encoded Boolean programs."""
    import torch
    n = int(lengths.numel())
    n_inputs = int(case_bits.shape[0]) if case_bits.dim() == 2 else 1
    if hits_out is None and out_words is None:
        hits_out = torch.empty(n, dtype=torch.int64, device=case_bits.device)
    _check(lib().gp_eval_population_bool_ex(_tptr(programs), _tptr(offsets), _tptr(lengths), n,
                                            _tptr(case_bits), n_inputs, int(n_cases),
                                            _tptr(target_bits), _tptr(hits_out),
                                            _tptr(out_words), _cfg(config), _stream(stream)))
    return hits_out


def eval_population_noalloc(programs, offsets, lengths, cases, targets, fitness_out=None,
                            stream=None):
    """gp_eval_population_noalloc: same result as eval_population, with the
    library's scratch in a fixed device array instead of allocated memory."""
    import torch
    n = int(lengths.numel())
    n_inputs, n_cases = (int(cases.shape[0]), int(cases.shape[1])) if cases.dim() == 2 else (1, int(cases.numel()))
    if fitness_out is None:
        fitness_out = torch.empty(n, dtype=torch.float64, device=cases.device)
    _check(lib().gp_eval_population_noalloc(_tptr(programs), _tptr(offsets), _tptr(lengths), n,
                                            _tptr(cases), n_inputs, n_cases, _tptr(targets),
                                            _tptr(fitness_out), _stream(stream)))
    return fitness_out


class _Segment(ctypes.Structure):
    _fields_ = [("prog_begin", ctypes.c_int32), ("n_progs", ctypes.c_int32), ("cases", ctypes.c_void_p),
                ("n_inputs", ctypes.c_int32), ("chunk", ctypes.c_int32), ("n_cases", ctypes.c_int64),
                ("targets", ctypes.c_void_p), ("out", ctypes.c_void_p)]


MAX_SEGMENTS = 64


def eval_segments(programs, offsets, lengths, segments, kind=None, config=None, stream=None):
    """gp_eval_segments: several populations in one launch.  `segments` is a
    list of dicts with prog_begin, n_progs, cases (CUDA tensor: float32
    [n_inputs, n_cases], or int32/uint32 bit words [n_inputs, n_words] with
    n_cases given), targets, out (float64 or int64 [n_progs]) and optionally
    chunk and n_cases.  kind: RUN_FLOAT (default) or RUN_BOOL."""
    kind = RUN_FLOAT if kind is None else kind
    arr = (_Segment * len(segments))()
    for i, g in enumerate(segments):
        x = g["cases"]
        n_inputs = int(x.shape[0]) if x.dim() == 2 else 1
        n_cases = int(g["n_cases"]) if "n_cases" in g else (int(x.shape[1]) if x.dim() == 2 else int(x.numel()))
        arr[i] = _Segment(int(g["prog_begin"]), int(g["n_progs"]), _tptr(x), n_inputs, int(g.get("chunk", 0)),
                          n_cases, _tptr(g["targets"]), _tptr(g["out"]))
    _check(lib().gp_eval_segments(_tptr(programs), _tptr(offsets), _tptr(lengths), arr, len(segments), kind,
                                  _cfg(config), _stream(stream)))


class Server:
    """gp_server_*: continuously batched evaluation of many GP runs' populations.

    Host numpy arrays in, host numpy arrays out; the server's own thread and
    streams do the device work.  Use as a context manager or call close().
    """

    def __init__(self, n_streams=4, max_inflight=16, max_queued=65536, max_merge=65536,
                 memory_budget=1 << 30, config: Optional[Config] = None):
        c = config or Config()
        opts = _ServerOpts(n_streams, max_inflight, max_queued, max_merge, memory_budget,
                           c.variant, c.k, c.block, 0, c.fitness, c.tile_inputs, c.stack_registers,
                           c.max_instructions)
        self._h = ctypes.c_void_p()
        _check(lib().gp_server_create(ctypes.byref(opts), ctypes.byref(self._h)))
        self._results = {}  # request id -> (buffer, keep-alive)

    def register_run(self, cases, targets, kind=RUN_FLOAT, n_cases=None) -> int:
        if kind == RUN_FLOAT:
            x = np.ascontiguousarray(cases, np.float32)
            x = x[None, :] if x.ndim == 1 else x
            y = np.ascontiguousarray(targets, np.float32)
            n_inputs, n = x.shape
        else:
            x = np.ascontiguousarray(cases, np.uint32)
            x = x[None, :] if x.ndim == 1 else x
            y = np.ascontiguousarray(targets, np.uint32)
            n_inputs, n = x.shape[0], int(n_cases)
        rid = ctypes.c_int32(-1)
        _check(lib().gp_server_register_run(self._h, kind, _np_ptr(x), n_inputs, n, _np_ptr(y),
                                            ctypes.byref(rid)))
        return int(rid.value)

    def submit(self, run_id: int, enc: "EncodedPopulation", n_nodes: Optional[int] = None,
               kind=RUN_FLOAT) -> int:
        n = enc.n
        out = np.zeros(n, np.float64 if kind == RUN_FLOAT else np.uint64)
        rid = ctypes.c_uint64(0)
        words = np.ascontiguousarray(enc.words, np.uint32)
        nodes = enc.nodes if n_nodes is None else n_nodes
        _check(lib().gp_server_submit(self._h, run_id, _np_ptr(words), _np_ptr(enc.offsets),
                                      _np_ptr(enc.lengths), n, nodes, _np_ptr(out),
                                      ctypes.byref(rid)))
        self._results[int(rid.value)] = out
        return int(rid.value)

    def wait(self, req_id: int, timeout_s: float = 60.0):
        """(result array, RequestInfo); raises GPError on timeout or failure."""
        info = RequestInfo()
        _check(lib().gp_server_wait(self._h, req_id, int(timeout_s * 1e6), ctypes.byref(info)))
        if info.status != 0:
            raise GPError(info.status, f"request {req_id} ended with status {info.status}")
        return self._results[req_id], info

    def poll(self, req_id: int):
        info = RequestInfo()
        rc = lib().gp_server_poll(self._h, req_id, ctypes.byref(info))
        if rc == 7:
            return None
        _check(rc)
        return info

    def cancel(self, req_id: int) -> int:
        return int(lib().gp_server_cancel(self._h, req_id))

    def stats(self) -> dict:
        st = ServerStats()
        _check(lib().gp_server_get_stats(self._h, ctypes.byref(st)))
        return st.as_dict()

    def close(self):
        if self._h:
            _check(lib().gp_server_destroy(self._h))
            self._h = ctypes.c_void_p()

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()


def autotune_population(programs, offsets, lengths, cases, targets, repeats=3, stream=None) -> Config:
    """gp_autotune_population: times k x block candidates on this workload and
    records the fastest for workloads of its shape; returns it."""
    n = int(lengths.numel())
    n_inputs, n_cases = (int(cases.shape[0]), int(cases.shape[1])) if cases.dim() == 2 else (1, int(cases.numel()))
    best = Config()
    _check(lib().gp_autotune_population(_tptr(programs), _tptr(offsets), _tptr(lengths), n,
                                        _tptr(cases), n_inputs, n_cases, _tptr(targets), repeats,
                                        ctypes.byref(best), _stream(stream)))
    return best


def autotune_population_ex(programs, offsets, lengths, cases, targets, base=None, repeats=3,
                           stream=None) -> Config:
    """gp_autotune_population_ex: times the candidates of the kernel family
    `base` names (Config or None for the default) and records the fastest."""
    n = int(lengths.numel())
    n_inputs, n_cases = (int(cases.shape[0]), int(cases.shape[1])) if cases.dim() == 2 else (1, int(cases.numel()))
    best = Config()
    _check(lib().gp_autotune_population_ex(_tptr(programs), _tptr(offsets), _tptr(lengths), n,
                                           _tptr(cases), n_inputs, n_cases, _tptr(targets), _cfg(base),
                                           repeats, ctypes.byref(best), _stream(stream)))
    return best


def autotune_population_bool(programs, offsets, lengths, case_bits, n_cases, target_bits, base=None,
                             repeats=3, stream=None) -> Config:
    """gp_autotune_population_bool: the same for a Boolean population."""
    n = int(lengths.numel())
    n_inputs = int(case_bits.shape[0]) if case_bits.dim() == 2 else 1
    best = Config()
    _check(lib().gp_autotune_population_bool(_tptr(programs), _tptr(offsets), _tptr(lengths), n,
                                             _tptr(case_bits), n_inputs, int(n_cases), _tptr(target_bits),
                                             _cfg(base), repeats, ctypes.byref(best), _stream(stream)))
    return best


def autotune_split_record(family, n_inputs, n_cases, n_progs):
    """gp_autotune_split_record: the width split the float tuner recorded for
    this shape, as (split_inputs, narrow Config, wide Config); split_inputs 0
    when none was recorded."""
    th = ctypes.c_int32(0)
    narrow, wide = Config(), Config()
    _check(lib().gp_autotune_split_record(int(family), int(n_inputs), int(n_cases), int(n_progs),
                                          ctypes.byref(th), ctypes.byref(narrow), ctypes.byref(wide)))
    return int(th.value), narrow, wide


def autotune_save(path: str):
    _check(lib().gp_autotune_save(os.fsencode(path)))


def autotune_load(path: str):
    _check(lib().gp_autotune_load(os.fsencode(path)))


def autotune_clear():
    _check(lib().gp_autotune_clear())


def set_config(variant=VARIANT_REGISTER, k=8, block=128, fitness=FITNESS_SUM_ABS, config=None):
    """gp_set_config: the default configuration (`config`, a Config, wins over
    the other arguments)."""
    c = config if config is not None else Config(variant, k, block, 0, fitness)
    _check(lib().gp_set_config(ctypes.byref(c)))


def reset_config():
    """gp_set_config(NULL): back to the library's own defaults."""
    _check(lib().gp_set_config(None))


def get_config() -> Config:
    c = Config()
    _check(lib().gp_get_config(ctypes.byref(c)))
    return c


def eval_launches(n_progs: int, n_cases: int) -> int:
    """Kernels one evaluation of n_progs programs over n_cases cases launches
    (the interpreter, and the longest-first ordering kernel for large
    populations over many cases)."""
    v = ctypes.c_int32(0)
    _check(lib().gp_eval_launches(int(n_progs), int(n_cases), ctypes.byref(v)))
    return int(v.value)


def last_error(stream=None) -> int:
    v = ctypes.c_int32(0)
    _check(lib().gp_last_error(_stream(stream), ctypes.byref(v)))
    return int(v.value)


def shutdown():
    _check(lib().gp_shutdown())


# ---------------------------------------------------------------------------
# device-side encoder and the on-device generation loop
# ---------------------------------------------------------------------------
def encode_slots_device(lengths, stream=None):
    """gp_encode_slots_device on a CUDA int32 tensor of tree lengths: the
    int64 offsets of back-to-back slots of 4 + 4 * lengths[p] words."""
    import torch
    n = int(lengths.numel())
    out_off = torch.empty(n, dtype=torch.int64, device=lengths.device)
    _check(lib().gp_encode_slots_device(_tptr(lengths), n, _tptr(out_off), _stream(stream)))
    return out_off


def encode_population_device(words, offsets, lengths, order: int = ORDER_MIN_DEPTH, stream=None):
    """gp_encode_population_device on CUDA tensors (user-format trees).
    Returns (out words, out offsets, out lengths) as CUDA tensors; program p
    is written at out_offsets[p], slots laid out back to back with room for
    4 + 4 * lengths[p] words."""
    import torch
    n = int(lengths.numel())
    out_off = encode_slots_device(lengths, stream)
    total = int((4 + 4 * lengths.to(torch.int64).clamp_min(0)).sum().item()) if n else 4
    out = torch.zeros(max(total, 4), dtype=torch.int32, device=lengths.device)
    out_len = torch.zeros(n, dtype=torch.int32, device=lengths.device)
    _check(lib().gp_encode_population_device(_tptr(words), _tptr(offsets), _tptr(lengths), n, order,
                                             _tptr(out), _tptr(out_off), _tptr(out_len),
                                             _stream(stream)))
    return out, out_off, out_len


class EvolveParams(ctypes.Structure):
    """gp_evolve_params (include/gpeval.h)."""
    _fields_ = [("pop_size", ctypes.c_int32), ("max_nodes", ctypes.c_int32),
                ("tournament", ctypes.c_int32), ("p_crossover", ctypes.c_float),
                ("p_mutation", ctypes.c_float), ("mutation_depth", ctypes.c_int32),
                ("n_funcs", ctypes.c_int32), ("funcs", ctypes.c_int32 * 16),
                ("p_const", ctypes.c_float), ("const_lo", ctypes.c_float),
                ("const_hi", ctypes.c_float), ("seed", ctypes.c_uint64), ("eval", Config)]

    @classmethod
    def make(cls, pop_size, funcs, max_nodes=255, tournament=7, p_crossover=0.95, p_mutation=0.2,
             mutation_depth=4, p_const=0.5, const_lo=-1.0, const_hi=1.0, seed=1, config=None):
        p = cls()
        p.pop_size, p.max_nodes, p.tournament = pop_size, max_nodes, tournament
        p.p_crossover, p.p_mutation, p.mutation_depth = p_crossover, p_mutation, mutation_depth
        p.n_funcs = len(funcs)
        for i, f in enumerate(funcs):
            p.funcs[i] = int(f)
        p.p_const, p.const_lo, p.const_hi, p.seed = p_const, const_lo, const_hi, seed
        if config is not None:
            p.eval = config
        return p


class Evolver:
    """gp_evolve_*: a GP run whose generations (variation, device encoding,
    evaluation) run on the GPU as CUDA-graph replays.  The initial population
    is host user-format trees; cases and targets are CUDA tensors kept alive
    by the run."""

    def __init__(self, params: EvolveParams, words, offsets, lengths, cases, targets):
        w = np.ascontiguousarray(words, np.uint32)
        off = np.ascontiguousarray(offsets, np.int64)
        ln = np.ascontiguousarray(lengths, np.int32)
        if ln.size != params.pop_size:
            raise ValueError("the initial population must have pop_size trees")
        self.params = params
        self._keep = (cases, targets)
        n_inputs, n_cases = (int(cases.shape[0]), int(cases.shape[1])) if cases.dim() == 2 else (1, int(cases.numel()))
        self._h = ctypes.c_void_p()
        _check(lib().gp_evolve_create(ctypes.byref(params), _np_ptr(w), _np_ptr(off), _np_ptr(ln),
                                      _tptr(cases), n_inputs, n_cases, _tptr(targets),
                                      ctypes.byref(self._h)))
        self.slot = 2 * params.max_nodes

    def run(self, generations: int = 1):
        _check(lib().gp_evolve_run(self._h, int(generations)))

    def read(self):
        """(list of token arrays, fitness float64 [n], generation index)."""
        n = self.params.pop_size
        words = np.zeros(n * self.slot, np.uint32)
        lens = np.zeros(n, np.int32)
        fit = np.zeros(n, np.float64)
        gen = ctypes.c_int32(0)
        _check(lib().gp_evolve_read(self._h, _np_ptr(words), _np_ptr(lens), _np_ptr(fit),
                                    ctypes.byref(gen), None))
        trees = [words[p * self.slot: p * self.slot + lens[p]].copy() for p in range(n)]
        return trees, fit, int(gen.value)

    def nodes_evaluated(self) -> int:
        """Tree nodes evaluated over all generations so far (waits for the run)."""
        v = ctypes.c_int64(0)
        _check(lib().gp_evolve_read(self._h, None, None, None, None, ctypes.byref(v)))
        return int(v.value)

    def close(self):
        if self._h:
            lib().gp_evolve_destroy(self._h)
            self._h = ctypes.c_void_p()

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
