"""The library's autotuner picks a measured (k, block) for a workload shape;
later evaluations that leave k and block at 0 use it and match an explicit
evaluation with that configuration bit for bit."""
import numpy as np
import pytest

import oracle
import synth
import paper_1601_00221_gb300 as gp
from gpu_util import dev, upload, assert_fitness

pytestmark = pytest.mark.gpu


def test_autotune_records_and_applies_the_fastest_configuration():
    w = synth.regression_small(seed=401, n_progs=600, n_cases=20000)
    enc = gp.encode_population(w.pop.words, w.pop.offsets, w.pop.lengths)
    P, O, L = upload(enc)
    X, Y = dev(w.cases), dev(w.targets)
    gp.autotune_clear()
    best = gp.autotune_population(P, O, L, X, Y, repeats=2)
    assert best.k in (2, 4, 8) and best.block in (64, 128, 256)
    assert best.chunk_cases == 0 or best.chunk_cases % (best.k * best.block) == 0
    tuned = gp.eval_population(P, O, L, X, Y).cpu().numpy()  # default config -> the tuned one
    explicit = gp.eval_population(P, O, L, X, Y, config=gp.Config(gp.VARIANT_REGISTER, best.k,
                                                                    best.block,
                                                                    best.chunk_cases)).cpu().numpy()
    assert np.array_equal(tuned.view(np.uint64), explicit.view(np.uint64))
    assert_fitness(tuned, oracle.population_fitness(w.pop.words, w.pop.offsets, w.pop.lengths,
                                                    w.cases, w.targets))
    gp.autotune_clear()


@pytest.fixture()
def clean_records():
    gp.autotune_clear()
    gp.reset_config()
    yield
    gp.autotune_clear()
    gp.reset_config()


def test_tuned_families_register_file_extended_and_boolean(clean_records):
    """The tuner covers every kernel family: for register programs it may
    choose the register-file variant, for S-form trees the stack levels in
    registers; each tuned configuration runs through the records (no
    configuration given) and gives the oracle's results."""
    import torch
    # register programs: the register variant's family, both forms tried
    lw = synth.linear_workload(seed=402, n_progs=200, n_cases=16384)
    le = gp.encode_linear_population(lw.pop.instr, lw.pop.offsets, lw.pop.lengths)
    P, O, L = upload(le)
    X, Y = dev(lw.cases), dev(lw.targets)
    best = gp.autotune_population_ex(P, O, L, X, Y, repeats=1)
    assert best.variant in (gp.VARIANT_REGISTER, gp.VARIANT_REGISTER_FILE)
    f = gp.eval_population(P, O, L, X, Y).cpu().numpy()
    assert_fitness(f, oracle.linear_population_fitness(lw.pop.instr, lw.pop.offsets, lw.pop.lengths,
                                                       lw.cases, lw.targets), "tuned register programs")
    # extended trees, classification fitness: the extended family
    sw = synth.shuttle_like_problem(seed=403, n_progs=300, n_cases=9000)
    se = gp.encode_population(sw.pop.words, sw.pop.offsets, sw.pop.lengths)
    P, O, L = upload(se)
    X, Y = dev(sw.cases), dev(sw.targets)
    base = se.config(fitness=gp.FITNESS_CLASS)
    best = gp.autotune_population_ex(P, O, L, X, Y, base=base, repeats=1)
    assert best.variant == gp.VARIANT_EXTENDED and best.tile_inputs == base.tile_inputs
    f = gp.eval_population(P, O, L, X, Y, config=base).cpu().numpy()  # k, block 0: the record
    exp = oracle.fset_population_fitness(sw.pop.words, sw.pop.offsets, sw.pop.lengths, sw.cases, sw.targets,
                                         oracle.FIT_CLASS)
    assert np.array_equal(f, exp)
    # Boolean
    bw = synth.boolean_problem("mux", 11, seed=404, n_progs=300)
    be = gp.encode_population(bw.pop.words, bw.pop.offsets, bw.pop.lengths, gp.KIND_BOOL)
    P, O, L = upload(be)
    cb = dev(bw.case_bits.view(np.int32))
    tb = dev(bw.target_bits.view(np.int32))
    best = gp.autotune_population_bool(P, O, L, cb, bw.n_cases, tb, repeats=1)
    assert best.k in (1, 2, 4, 8)
    h = gp.eval_population_bool(P, O, L, cb, bw.n_cases, tb).cpu().numpy()
    assert np.array_equal(h, oracle.bool_population_hits(bw.pop.words, bw.pop.offsets, bw.pop.lengths,
                                                         bw.case_bits, bw.n_cases, bw.target_bits))


def test_sform_tuning_may_hold_fewer_stack_levels_in_registers(clean_records):
    """S-form trees at k = 8: the candidates include stack levels 4..7 in
    shared memory; whichever wins, the recorded configuration reproduces the
    explicit evaluation bit for bit."""
    w = synth.regression_small(seed=405, n_progs=700, n_cases=20000)
    enc = gp.encode_population(w.pop.words, w.pop.offsets, w.pop.lengths)
    P, O, L = upload(enc)
    X, Y = dev(w.cases), dev(w.targets)
    best = gp.autotune_population_ex(P, O, L, X, Y, repeats=1)
    assert best.stack_registers in (0, 4)
    assert best.variant == gp.VARIANT_REGISTER  # trees: the register-file form cannot run them
    tuned = gp.eval_population(P, O, L, X, Y).cpu().numpy()
    explicit = gp.eval_population(P, O, L, X, Y, config=best).cpu().numpy()
    assert np.array_equal(tuned.view(np.uint64), explicit.view(np.uint64))
