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
