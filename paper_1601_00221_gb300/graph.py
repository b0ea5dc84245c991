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
"""
from __future__ import annotations

import ctypes
from typing import Optional

import numpy as np

from . import (Config, KIND_SFORM, ORDER_MIN_DEPTH, VARIANT_REGISTER, _check, _stream, _tptr,
               encode_population, lib)


class GenerationGraph:
    def __init__(self, n_progs: int, max_tokens: int, cases, targets, config: Optional[Config] = None,
                 kind: int = KIND_SFORM, order: int = ORDER_MIN_DEPTH, device="cuda"):
        """n_progs: population size; max_tokens: the largest total number of
        user-format words of any population to be evaluated; cases/targets:
        host arrays, binary32 [n_inputs, n_cases] and [n_cases]."""
        import torch
        self.torch = torch
        self.n = int(n_progs)
        self.kind, self.order = kind, order
        self.device = torch.device(device)
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
        self.graph = None
        self.nodes = 0

    def _device_work(self):
        torch = self.torch
        self.d_words.copy_(self.h_words, non_blocking=True)
        self.d_off.copy_(self.h_off, non_blocking=True)
        self.d_len.copy_(self.h_len, non_blocking=True)
        _check(lib().gp_eval_population_ex(
            _tptr(self.d_words), _tptr(self.d_off), _tptr(self.d_len), self.n, _tptr(self.X),
            self.n_inputs, self.n_cases, _tptr(self.Y), _tptr(self.d_fit), None,
            ctypes.byref(self.cfg), _stream(torch.cuda.current_stream())))
        self.h_fit.copy_(self.d_fit, non_blocking=True)

    def _encode(self, words, offsets, lengths):
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

    def run(self, words, offsets, lengths) -> np.ndarray:
        """Fitness (host float64 [n_progs]) of one generation's population."""
        if self.graph is None:
            self.capture(words, offsets, lengths)
        if len(lengths) != self.n:
            raise ValueError("population size differs from the graph's")
        self._encode(words, offsets, lengths)
        self.graph.replay()
        self.torch.cuda.current_stream().synchronize()
        self.stream.synchronize()
        return self.h_fit.numpy().copy()
