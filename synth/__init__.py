"""Seeded synthetic workloads for GP population evaluation.

This module only draws random programs and fitness cases and packs them into
the user token format.  It contains none of the evaluation method's arithmetic
(no program is ever interpreted here), so both the CUDA library and the CPU
oracle can take their inputs from it.  Targets of the regression problems are
the problem definitions themselves (a fixed polynomial of the inputs), written
as plain numpy expressions.

Workload recipes (all seeded, numpy PCG64):

* regression trees -- ramped half-and-half (Koza), root depth 1, half "full"
  and half "grow" per depth; grow draws a terminal with probability 0.5 below
  the maximum depth (the root is always a function); functions uniform over
  {+,-,*,protected /}; terminals are an input (uniform index) or a constant
  U[-1,1] with probability 0.5 each; trees above the node cap are redrawn.
* fitness cases x ~ U[-1,1] (binary32); target of the 1-input problem is
  y = x^4 + x^3 + x^2 + x computed in binary32 as
  ((x*x)*(x*x) + (x*x)*x) + (x*x + x).
* Boolean problems -- all 2^k input combinations, bit-packed 32 cases per
  uint32 word (case c -> word c>>5, bit c&31; input i of case c is bit i of c);
  even-k-parity and k-multiplexer targets; random trees over
  {AND,OR,NAND,NOR} (+IF for multiplexers) drawn ramped half-and-half, with a
  full tree that exceeds the node cap replaced by a grow tree.
* register linear GP -- lengths U{16..128}, destination, operands and function
  uniform over 8 registers and {+,-,*,/}; inputs ~N(0,1); target a seeded
  random polynomial of total degree <= 3 in 8 variables (all 165 monomials,
  coefficients U[-1,1]) evaluated in binary64 and rounded once to binary32.
* the paper's float problems (Sec. 4.2), synthetic stand-ins of the same
  shape (the Shuttle and KDDcup data sets are not available):
  - sextic regression: x ~ U[-1,1], 100000 cases, y = x^6 - 2x^4 + x^2
    (binary64, rounded once); trees over {*,/,+,-,sin,cos,log,exp} with
    terminals {x, U[-1,1] constants}; fitness mean squared error.
  - Shuttle-shaped classification (a full tree over the node cap -- IF has
    three children -- is replaced by a grow tree, as for the multiplexers):
    9 integer-valued inputs U{-100..100},
    58000 cases, 10 class labels 1..10 with 75% of the cases in class 1 (the
    rest uniform); trees over {*,/,+,-,>,<,==,AND,OR,IF}, constants
    U[-200,200]; fitness = incorrect classifications.
  - KDDcup-shaped classification: 41 inputs (a third integer counts
    floor(Exp(mean 100)), a third rates in [0,1] in steps of 0.01, a third
    0/1 flags), 494021 cases, 22 labels 0..21 with P(label i) proportional to
    2^-i; trees over all 14 functions, constants U[-20000,20000].
"""
from __future__ import annotations

from dataclasses import dataclass, field
from typing import List, Sequence

import numpy as np

# user token format: bits 0..7 opcode, bits 8..31 operand; CONST is followed
# by one word with the binary32 bit pattern of the constant.
ADD, SUB, MUL, DIV, VAR, CONST, AND, OR, NAND, NOR, IF = range(1, 12)
SIN, COS, EXP, LOG, GT, LT, EQ = range(12, 19)
FLOAT_FUNCS = (ADD, SUB, MUL, DIV)
BOOL_FUNCS = (AND, OR, NAND, NOR)
# the float function sets of Sec. 4.2 (AND, OR, IF act on floats in float trees)
SEXTIC_FUNCS = (MUL, DIV, ADD, SUB, SIN, COS, LOG, EXP)
SHUTTLE_FUNCS = (MUL, DIV, ADD, SUB, GT, LT, EQ, AND, OR, IF)
KDD_FUNCS = (ADD, SUB, MUL, DIV, GT, LT, EQ, AND, OR, IF, SIN, COS, LOG, EXP)
ARITY = {ADD: 2, SUB: 2, MUL: 2, DIV: 2, AND: 2, OR: 2, NAND: 2, NOR: 2, IF: 3,
         SIN: 1, COS: 1, EXP: 1, LOG: 1, GT: 2, LT: 2, EQ: 2}


def tok(op: int, arg: int = 0) -> int:
    return (op & 0xFF) | (arg << 8)


def const_tokens(v: float) -> List[int]:
    return [tok(CONST), int(np.float32(v).view(np.uint32))]


# --------------------------------------------------------------------------
# tree generation
# --------------------------------------------------------------------------
class _TreeGen:
    def __init__(self, rng, funcs, n_inputs, p_const, const_lo, const_hi):
        self.rng = rng
        self.funcs = tuple(funcs)
        self.n_inputs = n_inputs
        self.p_const = p_const
        self.const_lo = const_lo
        self.const_hi = const_hi

    def terminal(self, out: List[int]) -> int:
        if self.p_const > 0 and self.rng.random() < self.p_const:
            v = np.float32(self.rng.uniform(self.const_lo, self.const_hi))
            out.extend(const_tokens(float(v)))
        else:
            out.append(tok(VAR, int(self.rng.integers(0, self.n_inputs))))
        return 1

    def node(self, out: List[int], depth: int, max_depth: int, full: bool) -> int:
        if depth >= max_depth:
            return self.terminal(out)
        if not full and depth > 1 and self.rng.random() < 0.5:
            return self.terminal(out)
        f = self.funcs[int(self.rng.integers(0, len(self.funcs)))]
        out.append(tok(f))
        n = 1
        for _ in range(ARITY[f]):
            n += self.node(out, depth + 1, max_depth, full)
        return n


class _Uniforms:
    """U[0, 1) draws taken from blocks of a numpy generator (a few hundred
    nanoseconds per draw instead of a generator call per draw)."""

    def __init__(self, rng, block: int = 1 << 16):
        self.rng, self.block = rng, block
        self.buf, self.i = rng.random(block), 0

    def random(self) -> float:
        if self.i == self.block:
            self.buf, self.i = self.rng.random(self.block), 0
        v = self.buf[self.i]
        self.i += 1
        return float(v)

    def integers(self, lo: int, hi: int) -> int:
        return lo + min(int(self.random() * (hi - lo)), hi - lo - 1)

    def uniform(self, lo: float, hi: float) -> float:
        return lo + (hi - lo) * self.random()


def ramped_half_and_half(seed: int, n: int, depth_lo: int, depth_hi: int, max_nodes: int,
                         funcs: Sequence[int] = FLOAT_FUNCS, n_inputs: int = 1,
                         p_const: float = 0.5, const_lo: float = -1.0, const_hi: float = 1.0,
                         full_fallback_to_grow: bool = False, min_nodes: int = 1,
                         block_draws: bool = False) -> List[np.ndarray]:
    """n prefix trees; program i uses depth depth_lo + (i // 2) % span, full if i is even;
    trees outside [min_nodes, max_nodes] nodes are drawn again.  block_draws:
    the same distribution from blocks of uniform draws (much faster; other
    trees than the default for the same seed)."""
    rng = np.random.default_rng(seed)
    g = _TreeGen(_Uniforms(rng) if block_draws else rng, funcs, n_inputs, p_const, const_lo, const_hi)
    span = depth_hi - depth_lo + 1
    progs = []
    for i in range(n):
        d = depth_lo + (i // 2) % span
        full = (i % 2 == 0)
        for attempt in range(1000):
            out: List[int] = []
            use_full = full and not (full_fallback_to_grow and attempt > 0)
            nodes = g.node(out, 1, d, use_full)
            if min_nodes <= nodes <= max_nodes:
                break
        else:  # pragma: no cover - the caps used by the configs always fit
            raise RuntimeError("could not draw a tree under the node cap")
        progs.append(np.asarray(out, dtype=np.uint32))
    return progs


def count_nodes(prog: np.ndarray) -> int:
    """Nodes of a prefix token array (a CONST's payload word is not a node)."""
    n, i = 0, 0
    p = np.asarray(prog, dtype=np.uint32)
    while i < p.size:
        n += 1
        i += 2 if (int(p[i]) & 0xFF) == CONST else 1
    return n


@dataclass
class Population:
    words: np.ndarray           # uint32, all programs back to back
    offsets: np.ndarray         # int64 [n] word offset of program p
    lengths: np.ndarray         # int32 [n] words of program p
    nodes: np.ndarray           # int64 [n] tree nodes (GPop counting unit)

    @property
    def n(self) -> int:
        return int(self.lengths.size)

    def program(self, p: int) -> np.ndarray:
        o = int(self.offsets[p])
        return self.words[o:o + int(self.lengths[p])]


def pack(programs: Sequence[np.ndarray]) -> Population:
    lengths = np.array([len(p) for p in programs], dtype=np.int32)
    offsets = np.zeros(len(programs), dtype=np.int64)
    if len(programs) > 1:
        offsets[1:] = np.cumsum(lengths[:-1], dtype=np.int64)
    words = (np.concatenate([np.asarray(p, np.uint32) for p in programs])
             if programs else np.zeros(0, np.uint32))
    nodes = np.array([count_nodes(p) for p in programs], dtype=np.int64)
    return Population(words.astype(np.uint32), offsets, lengths, nodes)


# --------------------------------------------------------------------------
# regression cases
# --------------------------------------------------------------------------
def uniform_cases(seed: int, n_inputs: int, n_cases: int, lo=-1.0, hi=1.0) -> np.ndarray:
    rng = np.random.default_rng(seed)
    return rng.uniform(lo, hi, size=(n_inputs, n_cases)).astype(np.float32)


def quartic_target(x: np.ndarray) -> np.ndarray:
    """y = x^4 + x^3 + x^2 + x in binary32, grouped ((x*x)*(x*x) + (x*x)*x) + (x*x + x)."""
    x = np.asarray(x, np.float32)
    xx = x * x
    return ((xx * xx + xx * x) + (xx + x)).astype(np.float32)


def quartic_program() -> np.ndarray:
    """Prefix tokens of the tree that quartic_target writes out, input 0 = x."""
    X = tok(VAR, 0)
    xx = [tok(MUL), X, X]
    t = ([tok(ADD), tok(ADD), tok(MUL)] + xx + xx + [tok(MUL)] + xx + [X]
         + [tok(ADD)] + xx + [X])
    return np.asarray(t, np.uint32)


# --------------------------------------------------------------------------
# Boolean problems (bit-packed, 32 cases per word)
# --------------------------------------------------------------------------
def bool_case_bits(k: int) -> np.ndarray:
    """[k, n_words] uint32: bit (c & 31) of word (c >> 5) of row i is bit i of case c."""
    n_cases = 1 << k
    n_words = (n_cases + 31) // 32
    c = np.arange(n_words * 32, dtype=np.uint64)
    out = np.zeros((k, n_words), dtype=np.uint32)
    for i in range(k):
        bits = ((c >> np.uint64(i)) & np.uint64(1)).astype(np.uint32)
        bits[n_cases:] = 0
        out[i] = pack_bits(bits)
    return out


def pack_bits(bits: np.ndarray) -> np.ndarray:
    """Pack a 0/1 array (length multiple of 32 after zero padding) LSB first."""
    b = np.asarray(bits, np.uint32)
    pad = (-b.size) % 32
    if pad:
        b = np.concatenate([b, np.zeros(pad, np.uint32)])
    b = b.reshape(-1, 32)
    weights = (np.uint32(1) << np.arange(32, dtype=np.uint32))
    return (b * weights).sum(axis=1, dtype=np.uint64).astype(np.uint32)


def even_parity_target(k: int) -> np.ndarray:
    c = np.arange(1 << k, dtype=np.uint64)
    pc = np.zeros(c.size, np.uint32)
    for i in range(k):
        pc += ((c >> np.uint64(i)) & np.uint64(1)).astype(np.uint32)
    return pack_bits((pc % 2 == 0).astype(np.uint32))


def mux_address_bits(k: int) -> int:
    for a in range(1, 6):
        if a + (1 << a) == k:
            return a
    raise ValueError(f"{k} is not a multiplexer size a + 2^a")


def mux_target(k: int) -> np.ndarray:
    a = mux_address_bits(k)
    c = np.arange(1 << k, dtype=np.uint64)
    addr = np.zeros(c.size, np.uint64)
    for i in range(a):
        addr |= ((c >> np.uint64(i)) & np.uint64(1)) << np.uint64(i)
    out = (c >> (np.uint64(a) + addr)) & np.uint64(1)
    return pack_bits(out.astype(np.uint32))


# --------------------------------------------------------------------------
# register linear GP
# --------------------------------------------------------------------------
@dataclass
class LinearPopulation:
    instr: np.ndarray    # uint8 [total, 4] rows (dst, op, a, b)
    offsets: np.ndarray  # int64 [n] instruction offset
    lengths: np.ndarray  # int32 [n] instructions

    @property
    def n(self) -> int:
        return int(self.lengths.size)

    def program(self, p: int) -> np.ndarray:
        o = int(self.offsets[p])
        return self.instr[o:o + int(self.lengths[p])]


def linear_programs(seed: int, n: int, len_lo: int = 16, len_hi: int = 128,
                    n_regs: int = 8, funcs: Sequence[int] = FLOAT_FUNCS) -> LinearPopulation:
    rng = np.random.default_rng(seed)
    lengths = rng.integers(len_lo, len_hi + 1, size=n).astype(np.int32)
    total = int(lengths.sum())
    instr = np.empty((total, 4), np.uint8)
    instr[:, 0] = rng.integers(0, n_regs, size=total)
    instr[:, 1] = np.asarray(funcs, np.uint8)[rng.integers(0, len(funcs), size=total)]
    instr[:, 2] = rng.integers(0, n_regs, size=total)
    instr[:, 3] = rng.integers(0, n_regs, size=total)
    offsets = np.zeros(n, np.int64)
    if n > 1:
        offsets[1:] = np.cumsum(lengths[:-1], dtype=np.int64)
    return LinearPopulation(instr, offsets, lengths)


def normal_cases(seed: int, n_inputs: int, n_cases: int) -> np.ndarray:
    rng = np.random.default_rng(seed)
    return rng.standard_normal(size=(n_inputs, n_cases)).astype(np.float32)


def poly3_target(x: np.ndarray, seed: int) -> np.ndarray:
    """Random polynomial of total degree <= 3 in all rows of x (165 monomials for
    8 inputs), coefficients U[-1,1], evaluated in binary64, rounded once."""
    x = np.asarray(x, np.float64)
    nv = x.shape[0]
    rng = np.random.default_rng(seed)
    monos = [()]
    monos += [(i,) for i in range(nv)]
    monos += [(i, j) for i in range(nv) for j in range(i, nv)]
    monos += [(i, j, k) for i in range(nv) for j in range(i, nv) for k in range(j, nv)]
    coef = rng.uniform(-1.0, 1.0, size=len(monos))
    y = np.zeros(x.shape[1], np.float64)
    for c, m in zip(coef, monos):
        t = np.full(x.shape[1], c)
        for i in m:
            t = t * x[i]
        y += t
    return y.astype(np.float32)


# --------------------------------------------------------------------------
# the benchmark workloads
# --------------------------------------------------------------------------
@dataclass
class RegressionWorkload:
    name: str
    pop: Population
    cases: np.ndarray      # float32 [n_inputs, n_cases]
    targets: np.ndarray    # float32 [n_cases]
    meta: dict = field(default_factory=dict)

    @property
    def gpop(self) -> int:
        return int(self.pop.nodes.sum()) * int(self.cases.shape[1])


def regression_small(seed: int = 1, n_progs: int = 256, n_cases: int = 1024) -> RegressionWorkload:
    """256 ramped half-and-half trees (depth 2-6, <= 64 nodes), 1024 cases, quartic target."""
    progs = ramped_half_and_half(seed, n_progs, 2, 6, 64)
    x = uniform_cases(seed + 1000, 1, n_cases)
    return RegressionWorkload("regression-256x1024", pack(progs), x, quartic_target(x[0]),
                              {"depth": "2-6", "max_nodes": 64})


def regression_large(seed: int = 2, n_progs: int = 4096, n_cases: int = 65536) -> RegressionWorkload:
    """4096 ramped half-and-half trees (depth 2-8, <= 256 nodes), 65536 cases, quartic target."""
    progs = ramped_half_and_half(seed, n_progs, 2, 8, 256)
    x = uniform_cases(seed + 1000, 1, n_cases)
    return RegressionWorkload(f"regression-{n_progs}x{n_cases}", pack(progs), x,
                              quartic_target(x[0]), {"depth": "2-8", "max_nodes": 256})


@dataclass
class BooleanWorkload:
    name: str
    pop: Population
    case_bits: np.ndarray   # uint32 [k, n_words]
    target_bits: np.ndarray  # uint32 [n_words]
    n_cases: int

    @property
    def gpop(self) -> int:
        return int(self.pop.nodes.sum()) * self.n_cases


def boolean_problem(kind: str, k: int, seed: int = 3, n_progs: int = 4096,
                    max_nodes: int = 256) -> BooleanWorkload:
    """kind 'parity' (even-k-parity, {AND,OR,NAND,NOR}) or 'mux' (k-multiplexer, +IF)."""
    funcs = BOOL_FUNCS + ((IF,) if kind == "mux" else ())
    progs = ramped_half_and_half(seed, n_progs, 2, 8, max_nodes, funcs=funcs, n_inputs=k,
                                 p_const=0.0, full_fallback_to_grow=True)
    target = even_parity_target(k) if kind == "parity" else mux_target(k)
    return BooleanWorkload(f"{kind}{k}", pack(progs), bool_case_bits(k), target, 1 << k)


@dataclass
class LinearWorkload:
    name: str
    pop: LinearPopulation
    cases: np.ndarray
    targets: np.ndarray

    @property
    def gpop(self) -> int:
        return int(self.pop.lengths.sum()) * int(self.cases.shape[1])


def linear_workload(seed: int = 4, n_progs: int = 8192, n_cases: int = 262144,
                    len_lo: int = 16, len_hi: int = 128) -> LinearWorkload:
    pop = linear_programs(seed, n_progs, len_lo, len_hi)
    x = normal_cases(seed + 1000, 8, n_cases)
    return LinearWorkload(f"linear-{n_progs}x{n_cases}", pop, x, poly3_target(x, seed + 2000))


# --------------------------------------------------------------------------
# serving: many independent GP runs submitting populations
# --------------------------------------------------------------------------
@dataclass
class ServingRun:
    kind: str              # "float" or "bool"
    pop: Population
    cases: np.ndarray      # float32 [n_inputs, n_cases] or uint32 [n_inputs, n_words]
    targets: np.ndarray
    n_cases: int

    @property
    def gpop(self) -> int:
        return int(self.pop.nodes.sum()) * self.n_cases


def _serving_run(spec) -> ServingRun:
    """One serving run from its drawn parameters (a worker process may build it)."""
    kind, n_progs, s, lg, k, n_inputs, max_depth, max_nodes, min_nodes = spec
    if kind in ("mux", "parity"):
        funcs = BOOL_FUNCS + ((IF,) if kind == "mux" else ())
        progs = ramped_half_and_half(s, n_progs, 4, max_depth, max_nodes, funcs=funcs,
                                     n_inputs=k, p_const=0.0, full_fallback_to_grow=True,
                                     min_nodes=min_nodes, block_draws=True)
        target = even_parity_target(k) if kind == "parity" else mux_target(k)
        return ServingRun("bool", pack(progs), bool_case_bits(k), target, 1 << k)
    n_cases = 1 << lg
    progs = ramped_half_and_half(s, n_progs, 4, max_depth, max_nodes, n_inputs=n_inputs,
                                 min_nodes=min_nodes, block_draws=True)
    if n_inputs == 1:
        x = uniform_cases(s + 1, 1, n_cases)
        y = quartic_target(x[0])
    else:
        x = normal_cases(s + 1, 8, n_cases)
        y = poly3_target(x, s + 2)
    return ServingRun("float", pack(progs), x, y, n_cases)


def serving_runs(seed: int = 5, n_runs: int = 64, pop_lo: int = 128, pop_hi: int = 8192,
                 max_depth: int = 9, max_nodes: int = 512, log2_cases_lo: int = 10,
                 log2_cases_hi: int = 20, p_bool: float = 0.25, min_nodes: int = 8,
                 workers: int = 0) -> List[ServingRun]:
    """Independent runs of mixed kinds: float regression with 1 input (quartic
    target) or 8 inputs (random cubic target), and Boolean k-multiplexer or
    even-k-parity; population sizes U{pop_lo..pop_hi}; trees ramped
    half-and-half of depth 4..max_depth with min_nodes..max_nodes nodes; case
    counts 2^U{lo..hi} (Boolean: k inputs, 2^k cases with k in the same
    range).  workers > 1 builds the runs in that many spawned processes (the
    same runs as one process builds)."""
    rng = np.random.default_rng(seed)
    specs = []
    for r in range(n_runs):
        n_progs = int(rng.integers(pop_lo, pop_hi + 1))
        s = int(rng.integers(0, 2**31 - 1))
        lg = int(rng.integers(log2_cases_lo, log2_cases_hi + 1))
        if rng.random() < p_bool:
            kind = "mux" if rng.random() < 0.5 else "parity"
            k = lg
            if kind == "mux":  # nearest multiplexer size a + 2^a within the range
                k = min((a + (1 << a) for a in range(2, 5)), key=lambda v: abs(v - lg))
            specs.append((kind, n_progs, s, lg, k, k, max_depth, max_nodes, min_nodes))
        else:
            n_inputs = 1 if rng.random() < 0.5 else 8
            specs.append(("float", n_progs, s, lg, 0, n_inputs, max_depth, max_nodes, min_nodes))
    if workers > 1:
        import concurrent.futures as cf
        import multiprocessing as mp
        # largest first, so that the pool's last tasks are short
        by_size = sorted(range(n_runs), key=lambda i: -specs[i][1])
        with cf.ProcessPoolExecutor(max_workers=workers, mp_context=mp.get_context("spawn")) as ex:
            built = dict(zip(by_size, ex.map(_serving_run, [specs[i] for i in by_size])))
        return [built[i] for i in range(n_runs)]
    return [_serving_run(sp) for sp in specs]


# --------------------------------------------------------------------------
# the paper's float problems (Sec. 4.2), synthetic stand-ins
# --------------------------------------------------------------------------
def sextic_target(x: np.ndarray) -> np.ndarray:
    """x^6 - 2x^4 + x^2 in binary64, rounded once to binary32."""
    x64 = np.asarray(x, np.float64)
    return (x64 ** 6 - 2.0 * x64 ** 4 + x64 ** 2).astype(np.float32)


@dataclass
class FunctionSetWorkload:
    name: str
    pop: Population
    cases: np.ndarray       # float32 [n_inputs, n_cases]
    targets: np.ndarray     # float32 [n_cases] (class labels for classification)
    fitness: int            # 0 sum |e|, 1 mean squared error, 2 incorrect classifications
    funcs: tuple

    @property
    def gpop(self) -> float:
        return float(self.pop.nodes.sum()) * self.cases.shape[1]


def sextic_problem(seed: int = 6, n_progs: int = 4096, n_cases: int = 100000,
                   depth_lo: int = 2, depth_hi: int = 8, max_nodes: int = 256) -> FunctionSetWorkload:
    progs = ramped_half_and_half(seed, n_progs, depth_lo, depth_hi, max_nodes, funcs=SEXTIC_FUNCS)
    x = uniform_cases(seed + 1000, 1, n_cases)
    return FunctionSetWorkload("sextic", pack(progs), x, sextic_target(x[0]), 1, SEXTIC_FUNCS)


def shuttle_like_problem(seed: int = 7, n_progs: int = 4096, n_cases: int = 58000,
                         depth_lo: int = 2, depth_hi: int = 8,
                         max_nodes: int = 256) -> FunctionSetWorkload:
    progs = ramped_half_and_half(seed, n_progs, depth_lo, depth_hi, max_nodes, funcs=SHUTTLE_FUNCS,
                                 n_inputs=9, const_lo=-200.0, const_hi=200.0,
                                 full_fallback_to_grow=True)
    rng = np.random.default_rng(seed + 1000)
    x = rng.integers(-100, 101, (9, n_cases)).astype(np.float32)
    labels = np.where(rng.random(n_cases) < 0.75, 1, rng.integers(2, 11, n_cases)).astype(np.float32)
    return FunctionSetWorkload("shuttle-like", pack(progs), x, labels, 2, SHUTTLE_FUNCS)


def kdd_like_problem(seed: int = 8, n_progs: int = 1024, n_cases: int = 494021,
                     depth_lo: int = 2, depth_hi: int = 8,
                     max_nodes: int = 256) -> FunctionSetWorkload:
    progs = ramped_half_and_half(seed, n_progs, depth_lo, depth_hi, max_nodes, funcs=KDD_FUNCS,
                                 n_inputs=41, const_lo=-20000.0, const_hi=20000.0,
                                 full_fallback_to_grow=True)
    rng = np.random.default_rng(seed + 1000)
    x = np.empty((41, n_cases), np.float32)
    for v in range(41):
        if v % 3 == 0:
            x[v] = np.floor(rng.exponential(100.0, n_cases))
        elif v % 3 == 1:
            x[v] = rng.integers(0, 101, n_cases) / np.float32(100)
        else:
            x[v] = rng.integers(0, 2, n_cases)
    p = 2.0 ** -np.arange(22)
    labels = rng.choice(22, n_cases, p=p / p.sum()).astype(np.float32)
    return FunctionSetWorkload("kdd-like", pack(progs), x, labels, 2, KDD_FUNCS)
