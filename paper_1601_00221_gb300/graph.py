"""One GP generation's device work as a replayable CUDA graph.

A GP run evaluates a new population of the same size against the same
fitness cases every generation (Sec. 4.2: population 1000, 50 generations).
`GenerationGraph` keeps the cases resident, owns pinned host buffers and
device buffers sized for the population's largest encoding, and captures
once: copy the encoded programs host -> device, evaluate (gp_eval_population_ex
with a fixed configuration), copy the fitness device -> host.  Each generation
then only encodes into the pinned buffer on the host (multi-threaded C++
encoder) and replays the graph: one launch instead of five calls.

The graph copies the whole capacity of the program buffer every replay (the
size is fixed at capture); the words past the population's encoding are not
read by the kernel.

With `device_encode=True` the host encodes nothing: the graph copies the
user-format trees themselves and runs the device-side encoder
(gp_encode_population_device) before the evaluation, so the host's work per
generation is one copy of the trees into pinned memory (trees of at most
GP_DEVICE_ENCODE_MAX_NODES nodes, S-form).
"""
from __future__ import annotations

import ctypes
from typing import Optional

import numpy as np

from . import (Config, KIND_SFORM, ORDER_MIN_DEPTH, VARIANT_REGISTER, _check, _stream, _tptr,
               encode_population, lib)

DEVICE_ENCODE_MAX_NODES = 256  # GP_DEVICE_ENCODE_MAX_NODES


class GenerationGraph:
    def __init__(self, n_progs: int, max_tokens: int, cases, targets, config: Optional[Config] = None,
                 kind: int = KIND_SFORM, order: int = ORDER_MIN_DEPTH, device="cuda",
                 device_encode: bool = False, shared_cases: Optional["GenerationGraph"] = None):
        """n_progs: population size; max_tokens: the largest total number of
        user-format words of any population to be evaluated; cases/targets:
        host arrays, binary32 [n_inputs, n_cases] and [n_cases] (ignored when
        shared_cases, another graph on the same device, lends its resident
        copy)."""
        import torch
        self.torch = torch
        self.n = int(n_progs)
        self.kind, self.order = kind, order
        self.device_encode = bool(device_encode)
        if self.device_encode and kind != KIND_SFORM:
            raise ValueError("the device-side encoder writes the S-form only")
        self.max_tokens = int(max_tokens)
        self.device = torch.device(device)
        if shared_cases is not None:
            self.X, self.Y = shared_cases.X, shared_cases.Y
            self.n_inputs, self.n_cases = shared_cases.n_inputs, shared_cases.n_cases
        else:
            x = np.ascontiguousarray(cases, np.float32)
            x = x[None, :] if x.ndim == 1 else x
            self.n_inputs, self.n_cases = int(x.shape[0]), int(x.shape[1])
            self.X = torch.from_numpy(x).to(self.device)
            self.Y = torch.from_numpy(np.ascontiguousarray(targets, np.float32)).to(self.device)
        self.cap = 4 * self.n + 4 * int(max_tokens)
        pin = lambda n, dt: torch.empty(n, dtype=dt).pin_memory()
        self.h_words = pin(self.cap, torch.int32)
        self.h_off = pin(self.n, torch.int64)
        self.h_len = pin(self.n, torch.int32)
        self.h_fit = pin(self.n, torch.float64)
        self.d_words = torch.zeros(self.cap, dtype=torch.int32, device=self.device)
        self.d_off = torch.zeros(self.n, dtype=torch.int64, device=self.device)
        self.d_len = torch.full((self.n,), 4, dtype=torch.int32, device=self.device)
        self.d_fit = torch.empty(self.n, dtype=torch.float64, device=self.device)
        self.cfg = config or Config(VARIANT_REGISTER, 8, 256, 0)
        self.stream = torch.cuda.Stream(device=self.device)
        self.done = torch.cuda.Event()
        self.pending = False  # a replay whose fitness has not been collected
        self.graph = None
        self.nodes = 0
        if self.device_encode:
            # trees in; encoded programs in back-to-back slots of 4 + 4 * lengths[p]
            # words, laid out on the device (gp_encode_slots_device)
            self.h_tok = pin(max(self.max_tokens, 1), torch.int32)
            self.d_tok = torch.zeros(max(self.max_tokens, 1), dtype=torch.int32, device=self.device)
            self.d_eoff = torch.zeros(self.n, dtype=torch.int64, device=self.device)
            self.d_elen = torch.full((self.n,), 4, dtype=torch.int32, device=self.device)

    def _device_work(self):
        torch = self.torch
        stream = _stream(torch.cuda.current_stream())
        if self.device_encode:
            self.d_tok.copy_(self.h_tok, non_blocking=True)
            self.d_off.copy_(self.h_off, non_blocking=True)
            self.d_len.copy_(self.h_len, non_blocking=True)
            _check(lib().gp_encode_slots_device(_tptr(self.d_len), self.n, _tptr(self.d_eoff), stream))
            _check(lib().gp_encode_population_device(
                _tptr(self.d_tok), _tptr(self.d_off), _tptr(self.d_len), self.n, self.order,
                _tptr(self.d_words), _tptr(self.d_eoff), _tptr(self.d_elen), stream))
            words, off, ln = self.d_words, self.d_eoff, self.d_elen
        else:
            self.d_words.copy_(self.h_words, non_blocking=True)
            self.d_off.copy_(self.h_off, non_blocking=True)
            self.d_len.copy_(self.h_len, non_blocking=True)
            words, off, ln = self.d_words, self.d_off, self.d_len
        _check(lib().gp_eval_population_ex(
            _tptr(words), _tptr(off), _tptr(ln), self.n, _tptr(self.X), self.n_inputs,
            self.n_cases, _tptr(self.Y), _tptr(self.d_fit), None, ctypes.byref(self.cfg), stream))
        self.h_fit.copy_(self.d_fit, non_blocking=True)

    def _stage_trees(self, words, offsets, lengths):
        """Device encoding: the trees into pinned memory -- the caller's words
        as they are, with the caller's offsets, when they fit the capacity;
        else packed back to back."""
        w = np.ascontiguousarray(words, np.uint32)
        off = np.ascontiguousarray(offsets, np.int64)
        ln = np.ascontiguousarray(lengths, np.int32)
        tok = self.h_tok.numpy().view(np.uint32)
        n = ln.size
        lc = np.maximum(ln, 0)
        if int(lc.sum()) > self.max_tokens:  # the encoded slots' bound
            raise ValueError("the population has more words than the graph's capacity")
        if n and int(off.min()) < 0:
            raise ValueError("negative program offset")
        end = int((off + lc).max()) if n else 0
        if end > w.size:
            raise ValueError("a program runs past the end of the words")
        if end <= self.max_tokens:
            tok[:end] = w[:end]
            self.h_off.numpy()[:] = off
        else:
            pos = 0
            for p in range(n):
                k = int(lc[p])
                tok[pos:pos + k] = w[off[p]:off[p] + k]
                self.h_off.numpy()[p] = pos
                pos += k
        self.h_len.numpy()[:] = ln

    def _encode(self, words, offsets, lengths):
        if self.device_encode:
            self._stage_trees(words, offsets, lengths)
            return None
        out = self.h_words.numpy().view(np.uint32)
        enc = encode_population(words, offsets, lengths, self.kind, self.order, out=out)
        if enc.words.ctypes.data != out.ctypes.data:
            raise ValueError("population encoding does not fit the graph's capacity")
        self.h_off.numpy()[:] = enc.offsets
        self.h_len.numpy()[:] = enc.lengths
        self.nodes = enc.nodes
        return enc

    def capture(self, words, offsets, lengths):
        """Encodes a first population, runs it eagerly (sizing the library's
        workspace), then captures the generation step."""
        torch = self.torch
        if len(lengths) != self.n:
            raise ValueError("population size differs from the graph's")
        self._encode(words, offsets, lengths)
        with torch.cuda.stream(self.stream):
            self._device_work()
        self.stream.synchronize()
        self.graph = torch.cuda.CUDAGraph()
        with torch.cuda.graph(self.graph, stream=self.stream):
            self._device_work()
        return self

    def launch(self, words, offsets, lengths) -> None:
        """Stages one population into the pinned buffers and replays the graph
        on this graph's stream without waiting for it; `collect` returns its
        fitness.  A launch first waits for the previous replay of this graph
        (its pinned buffers are about to be overwritten); that replay's
        fitness must have been collected."""
        if self.pending:
            raise RuntimeError("collect the previous launch's fitness first")
        if self.graph is None:
            self.capture(words, offsets, lengths)
        elif len(lengths) != self.n:
            raise ValueError("population size differs from the graph's")
        else:
            self._encode(words, offsets, lengths)
        with self.torch.cuda.stream(self.stream):
            self.graph.replay()
            self.done.record(self.stream)
        self.pending = True

    def collect(self) -> np.ndarray:
        """Fitness (host float64 [n_progs]) of the last launch."""
        if not self.pending:
            raise RuntimeError("nothing launched")
        self.done.synchronize()
        self.pending = False
        return self.h_fit.numpy().copy()

    def run(self, words, offsets, lengths) -> np.ndarray:
        """Fitness (host float64 [n_progs]) of one generation's population."""
        self.launch(words, offsets, lengths)
        return self.collect()


class EvaluationPipeline:
    """Independent populations of one size (the generations of several GP
    runs, a queue of evaluation requests) through `depth` generation graphs
    in turn, each on its own stream: while one population evaluates, the
    host stages the next into another graph's pinned buffers and that
    graph's copy and device encoding run beside the evaluation, so a stream
    of populations approaches the evaluation's own rate.  Every population
    still crosses the host-device boundary both ways (trees in, fitness
    out).  The graphs share one resident copy of the cases.

        pipe = EvaluationPipeline(n, max_tokens, cases, targets, device_encode=True)
        for pop in populations:
            for ticket, fit in pipe.submit(pop.words, pop.offsets, pop.lengths):
                ...   # results that finished, in submission order
        for ticket, fit in pipe.drain():
            ...
    """

    def __init__(self, n_progs: int, max_tokens: int, cases, targets, depth: int = 2, **kwargs):
        if depth < 1:
            raise ValueError("depth must be at least 1")
        first = GenerationGraph(n_progs, max_tokens, cases, targets, **kwargs)
        self.graphs = [first] + [GenerationGraph(n_progs, max_tokens, None, None, shared_cases=first, **kwargs)
                                 for _ in range(depth - 1)]
        self.next_ticket = 0
        self.inflight = []  # (ticket, graph) in submission order

    def submit(self, words, offsets, lengths):
        """Launches one population; returns the (ticket, fitness) pairs of the
        populations that had to be collected to free a graph (at most one),
        oldest first.  Tickets count submissions from 0."""
        out = []
        g = self.graphs[self.next_ticket % len(self.graphs)]
        if g.pending:  # the oldest launch holds this graph
            t, og = self.inflight.pop(0)
            assert og is g
            out.append((t, g.collect()))
        g.launch(words, offsets, lengths)
        self.inflight.append((self.next_ticket, g))
        self.next_ticket += 1
        return out

    def drain(self):
        """(ticket, fitness) of every population still in flight, oldest first."""
        out = []
        while self.inflight:
            t, g = self.inflight.pop(0)
            out.append((t, g.collect()))
        return out
