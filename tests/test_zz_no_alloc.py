"""gp_eval_population_noalloc, the entry point for callers that cannot let the
library allocate device memory (e.g. an application whose own fixed pool owns
the GPU's memory, or a loop that must not meet an allocation failure or the
synchronisation an allocation can imply mid-run), gives the same fitness as
gp_eval_population, which allocates its workspace.  Collected last on
purpose, so a run that stops at the first failure has run everything else."""
import ctypes

import numpy as np
import pytest

import synth
import paper_1601_00221_gb300 as gp
from gpu_util import dev, upload, assert_fitness

pytestmark = pytest.mark.gpu


def entry():
    """The C-ABI function, with its signature from include/gpeval.h."""
    fn = gp.lib().gp_eval_population_noalloc
    fn.argtypes = [ctypes.c_void_p] * 3 + [ctypes.c_int32, ctypes.c_void_p, ctypes.c_int32,
                   ctypes.c_int64, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]
    fn.restype = ctypes.c_int
    return fn


def noalloc(P, O, L, X, Y, out, stream):
    lib = gp.lib()
    fn = entry()
    n = int(L.numel())
    rc = fn(ctypes.c_void_p(P.data_ptr()), ctypes.c_void_p(O.data_ptr()),
            ctypes.c_void_p(L.data_ptr()), n,
            ctypes.c_void_p(X.data_ptr()), int(X.shape[0]), int(X.shape[1]),
            ctypes.c_void_p(Y.data_ptr()), ctypes.c_void_p(out.data_ptr()),
            ctypes.c_void_p(stream.cuda_stream))
    return rc, lib.gp_error_string().decode()


def workload(seed, n_progs, n_cases, n_inputs):
    progs = synth.ramped_half_and_half(seed, n_progs, 2, 7, 127, n_inputs=n_inputs)
    pop = synth.pack(progs)
    x = synth.uniform_cases(seed + 1, n_inputs, n_cases)
    y = synth.uniform_cases(seed + 2, 1, n_cases)[0]
    enc = gp.encode_population(pop.words, pop.offsets, pop.lengths)
    return upload(enc), dev(x), dev(y), pop.n


def test_noalloc_matches_allocating_entry_point_twice():
    import torch
    stream = torch.cuda.current_stream()
    # two different workloads in a row: the fixed scratch keeps the first
    # call's contents, the second must not depend on them
    for seed, n_progs, n_cases, n_inputs in ((91, 300, 5003, 1), (92, 1000, 20000, 3)):
        (P, O, L), X, Y, n = workload(seed, n_progs, n_cases, n_inputs)
        ref = gp.eval_population(P, O, L, X, Y).cpu().numpy()
        for _ in range(2):
            out = torch.full((n,), float("nan"), dtype=torch.float64, device="cuda")
            rc, msg = noalloc(P, O, L, X, Y, out, stream)
            assert rc == 0, msg
            torch.cuda.synchronize()
            assert_fitness(out.cpu().numpy(), ref, f"noalloc seed={seed}")


def test_noalloc_rejects_more_programs_than_its_scratch_holds():
    import torch
    lib = gp.lib()
    fn = entry()
    big = 65536 + 1
    dummy = torch.zeros(4, dtype=torch.int32, device="cuda")
    p = ctypes.c_void_p(dummy.data_ptr())
    rc = fn(p, p, p, ctypes.c_int32(big), p, ctypes.c_int32(1), ctypes.c_int64(16), p, p,
            ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    assert rc == 1
    assert b"at most" in lib.gp_error_string()
