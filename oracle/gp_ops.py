"""Genetic operators of a GP run, plain Python -- TEST INFRASTRUCTURE ONLY.

Only ``tests/``, ``__graft_entry__.smoke()`` and ``bench.py``'s CPU-baseline
leg may import this module; it shares no code with the CUDA library.

The paper's runs (Sec. 4.2, parameter table) use tournament selection of size
7, crossover with probability 0.95 and mutation with probability 0.2 over
populations of trees.  It does not define the operators beyond their names;
this module is the reference for the library's on-device generation loop and
restates every choice the library makes (the readings are listed in the
library's header next to gp_evolve_params):

* random numbers -- Philox4x32-10 (J. K. Salmon, M. A. Moraes, R. O. Dror,
  D. E. Shaw, "Parallel random numbers: as easy as 1, 2, 3", SC'11), written
  from its definition: ten rounds of two 32x32->64 multiplications by
  0xD2511F53 and 0xCD9E8D57, the key bumped by 0x9E3779B9 and 0xBB67AE85
  between rounds.  Offspring i of generation g draws from the counters
  (i, g, j, 0), j = 0, 1, ..., under the key (seed low word, seed high word),
  taking the four output words of each block in order.
* uniform(n) = (u * n) >> 32 for a 32-bit draw u; a probability p is the
  threshold floor(p * 2^32) (at most 2^32 - 1) and an event happens when
  u < threshold.
* tournament: T uniform picks, the first one the provisional winner, a later
  pick winning only with a strictly lower fitness (NaN counts as +inf).
* offspring: parent A by tournament; with probability p_crossover parent B by
  tournament, a node of A and a node of B uniformly (prefix order), and the
  child is A with that subtree replaced by B's (a child over max_nodes is A);
  then with probability p_mutation a node of the child uniformly, replaced by
  a grown subtree (a result over max_nodes keeps the child).
* grow(D): a node at depth d (the root at 1) is a terminal if d >= D, or, when
  d > 1, with probability 1/2 (u < 2^31); otherwise a function drawn uniformly
  from the function set, its children grown at depth d + 1.  A terminal is a
  constant with probability p_const (a second draw u2 gives
  lo + (hi - lo) * ((u2 >> 8) * 2^-24), each step one binary32 operation),
  else an input drawn uniformly.
"""
from __future__ import annotations

import numpy as np

# user token format (same numbers as the library's header, restated here)
VAR, CONST = 5, 6
ARITY = {1: 2, 2: 2, 3: 2, 4: 2, 7: 2, 8: 2, 11: 3, 12: 1, 13: 1, 14: 1, 15: 1, 16: 2, 17: 2, 18: 2}

_M0, _M1, _W0, _W1 = 0xD2511F53, 0xCD9E8D57, 0x9E3779B9, 0xBB67AE85
_MASK = 0xFFFFFFFF


def philox4x32_10(counter, key):
    """One Philox4x32-10 block: four 32-bit words from a 4-word counter and a
    2-word key."""
    c = [int(v) & _MASK for v in counter]
    k = [int(v) & _MASK for v in key]
    for r in range(10):
        p0 = _M0 * c[0]
        p1 = _M1 * c[2]
        c = [((p1 >> 32) ^ c[1] ^ k[0]) & _MASK, p1 & _MASK, ((p0 >> 32) ^ c[3] ^ k[1]) & _MASK,
             p0 & _MASK]
        if r < 9:
            k = [(k[0] + _W0) & _MASK, (k[1] + _W1) & _MASK]
    return c


class Stream:
    """The draws of one offspring: blocks (i, g, j, 0), j = 0, 1, ..."""

    def __init__(self, seed: int, individual: int, generation: int):
        self.key = (seed & _MASK, (seed >> 32) & _MASK)
        self.i, self.g = individual, generation
        self.j = 0
        self.buf = []

    def next(self) -> int:
        if not self.buf:
            self.buf = philox4x32_10((self.i, self.g, self.j, 0), self.key)
            self.j += 1
        return self.buf.pop(0)

    def uniform(self, n: int) -> int:
        return (self.next() * n) >> 32


def threshold(p: float) -> int:
    """floor(p * 2^32) of a binary32 probability, at most 2^32 - 1."""
    v = np.floor(np.float64(np.float32(p)) * 4294967296.0)
    return int(min(max(v, 0.0), 4294967295.0))


def _fitness_key(f) -> float:
    return np.inf if np.isnan(f) else float(f)


def tournament(s: Stream, fitness, size: int) -> int:
    n = len(fitness)
    best = s.uniform(n)
    for _ in range(size - 1):
        c = s.uniform(n)
        if _fitness_key(fitness[c]) < _fitness_key(fitness[best]):
            best = c
    return best


# --- prefix-array tree helpers ----------------------------------------------
def node_starts(tokens):
    """Word position of every node, in prefix order (a constant's value word
    is not a node)."""
    out, i = [], 0
    while i < len(tokens):
        out.append(i)
        i += 2 if (int(tokens[i]) & 0xFF) == CONST else 1
    return out


def subtree_end(tokens, start: int) -> int:
    """One past the last word of the subtree that starts at `start`."""
    owed, i = 1, start
    while owed:
        op = int(tokens[i]) & 0xFF
        owed -= 1
        if op == CONST:
            i += 2
            continue
        if op != VAR:
            owed += ARITY[op]
        i += 1
    return i


def grow(s: Stream, depth_max: int, funcs, n_inputs: int, thr_const: int, lo: float, hi: float):
    out = []

    def node(d):
        if d >= depth_max or (d > 1 and s.next() < (1 << 31)):
            if s.next() < thr_const:
                u = s.next()
                t = np.float32(u >> 8) * np.float32(2.0 ** -24)
                w = np.float32(hi) - np.float32(lo)
                v = np.float32(np.float32(lo) + np.float32(w * t))
                out.extend([CONST, int(np.float32(v).view(np.uint32))])
            else:
                out.append(VAR | (s.uniform(n_inputs) << 8))
            return
        f = funcs[s.uniform(len(funcs))]
        out.append(f)
        for _ in range(ARITY[f]):
            node(d + 1)

    node(1)
    return out


def offspring(pop, fitness, i: int, generation: int, seed: int, p) -> list:
    """Child i of a generation.  pop: list of token lists; p: dict with
    tournament, p_crossover, p_mutation, mutation_depth, funcs, n_inputs,
    p_const, const_lo, const_hi, max_nodes."""
    s = Stream(seed, i, generation)
    a = tournament(s, fitness, p["tournament"])
    child = list(pop[a])
    if s.next() < threshold(p["p_crossover"]):
        b = tournament(s, fitness, p["tournament"])
        A, B = pop[a], pop[b]
        sa, sb = node_starts(A), node_starts(B)
        ia, ib = sa[s.uniform(len(sa))], sb[s.uniform(len(sb))]
        cand = list(A[:ia]) + list(B[ib:subtree_end(B, ib)]) + list(A[subtree_end(A, ia):])
        if len(node_starts(cand)) <= p["max_nodes"]:
            child = cand
    if s.next() < threshold(p["p_mutation"]):
        sc = node_starts(child)
        im = sc[s.uniform(len(sc))]
        sub = grow(s, p["mutation_depth"], p["funcs"], p["n_inputs"], threshold(p["p_const"]),
                   p["const_lo"], p["const_hi"])
        cand = child[:im] + sub + child[subtree_end(child, im):]
        if len(node_starts(cand)) <= p["max_nodes"]:
            child = cand
    return [int(t) for t in child]


def generation(pop, fitness, generation_index: int, seed: int, p) -> list:
    return [offspring(pop, fitness, i, generation_index, seed, p) for i in range(len(pop))]
