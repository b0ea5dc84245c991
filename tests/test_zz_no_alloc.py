"""gp_eval_population_noalloc, the entry point for callers that cannot let the
library allocate device memory (an application whose own fixed pool owns the
GPU's memory, or a loop that must not meet an allocation failure or the
synchronisation an allocation can imply mid-run), gives what
gp_eval_population gives -- bit for bit, since it runs the same kernel with
the same configuration and split of the cases -- and what the oracle gives,
within the fitness tolerance, on two calls in a row: under the three fitness
measures, with the extended interpreter, with no cases, and after the
autotuner has recorded a configuration.  Collected last on purpose, so a run
that stops at the first failure has run everything else; each test restores
the library's default configuration."""
import ctypes

import numpy as np
import pytest

import oracle
import synth
import paper_1601_00221_gb300 as gp
from gpu_util import dev, upload, assert_fitness

pytestmark = pytest.mark.gpu


@pytest.fixture(autouse=True)
def library_defaults():
    gp.reset_config()
    gp.autotune_clear()
    yield
    gp.reset_config()
    gp.autotune_clear()


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
    return pop, x, y


def twice_against(P, O, L, X, Y, n, ref, exp, what):
    """Two calls in a row: each bit-identical to the allocating entry point's
    fitness `ref` and within the tolerance of the oracle's `exp`."""
    import torch
    stream = torch.cuda.current_stream()
    for call in range(2):
        out = torch.full((n,), float("nan"), dtype=torch.float64, device="cuda")
        rc, msg = noalloc(P, O, L, X, Y, out, stream)
        assert rc == 0, msg
        torch.cuda.synchronize()
        got = out.cpu().numpy()
        assert np.array_equal(got.view(np.uint64), ref.view(np.uint64)), f"{what} call {call}: not bit-identical"
        assert_fitness(got, exp, f"{what} call {call} vs the oracle")


def test_noalloc_matches_allocating_entry_point_and_oracle_twice():
    # two different workloads in a row: the fixed scratch keeps the first
    # call's contents, the second must not depend on them
    for seed, n_progs, n_cases, n_inputs in ((91, 300, 5003, 1), (92, 1000, 20000, 3)):
        pop, x, y = workload(seed, n_progs, n_cases, n_inputs)
        enc = gp.encode_population(pop.words, pop.offsets, pop.lengths)
        P, O, L = upload(enc)
        X, Y = dev(x), dev(y)
        ref = gp.eval_population(P, O, L, X, Y).cpu().numpy()
        exp = oracle.population_fitness(pop.words, pop.offsets, pop.lengths, x, y)
        twice_against(P, O, L, X, Y, pop.n, ref, exp, f"seed={seed}")


@pytest.mark.parametrize("fit", [gp.FITNESS_SUM_ABS, gp.FITNESS_MSE, gp.FITNESS_CLASS])
def test_noalloc_fitness_measures_extended_interpreter(fit):
    # Shuttle-set trees (comparisons, AND, OR, IF: exact functions) with the
    # extended S-form interpreter, as the default configuration
    w = synth.shuttle_like_problem(seed=93, n_progs=200, n_cases=3001)
    enc = gp.encode_population(w.pop.words, w.pop.offsets, w.pop.lengths)
    gp.set_config(config=gp.Config(gp.VARIANT_EXTENDED, 4, 128, 0, fit))
    P, O, L = upload(enc)
    X, Y = dev(w.cases), dev(w.targets)
    ref = gp.eval_population(P, O, L, X, Y).cpu().numpy()
    exp = oracle.fset_population_fitness(w.pop.words, w.pop.offsets, w.pop.lengths, w.cases, w.targets, fit)
    twice_against(P, O, L, X, Y, w.pop.n, ref, exp, f"extended fit={fit}")


def test_noalloc_after_autotune_uses_the_recorded_configuration():
    pop, x, y = workload(94, 400, 40000, 1)
    enc = gp.encode_population(pop.words, pop.offsets, pop.lengths)
    P, O, L = upload(enc)
    X, Y = dev(x), dev(y)
    gp.autotune_population(P, O, L, X, Y, repeats=1)
    ref = gp.eval_population(P, O, L, X, Y).cpu().numpy()
    exp = oracle.population_fitness(pop.words, pop.offsets, pop.lengths, x, y)
    twice_against(P, O, L, X, Y, pop.n, ref, exp, "after autotune")


def test_noalloc_no_cases_gives_zero():
    import torch
    pop, _, _ = workload(95, 16, 1, 1)
    P, O, L = upload(gp.encode_population(pop.words, pop.offsets, pop.lengths))
    X = dev(np.zeros((1, 0), np.float32))
    Y = dev(np.zeros(0, np.float32))
    for fit in (gp.FITNESS_SUM_ABS, gp.FITNESS_MSE, gp.FITNESS_CLASS):
        gp.set_config(fitness=fit)
        out = torch.full((pop.n,), float("nan"), dtype=torch.float64, device="cuda")
        rc, msg = noalloc(P, O, L, X, Y, out, torch.cuda.current_stream())
        assert rc == 0, msg
        assert np.all(out.cpu().numpy() == 0.0)


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
    rc = fn(p, p, p, ctypes.c_int32(4), p, ctypes.c_int32(1), ctypes.c_int64((1 << 40) + 1), p, p,
            ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    assert rc == 1
    assert b"too large" in lib.gp_error_string()
