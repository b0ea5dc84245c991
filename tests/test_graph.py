"""A CUDA-graph generation step (host encoding into pinned memory, then one
graph replay: copy in, evaluate, copy out) gives the same fitness as the
direct evaluation, generation after generation."""
import numpy as np
import pytest

import synth
import paper_1601_00221_gb300 as gp
from paper_1601_00221_gb300.graph import GenerationGraph
from gpu_util import dev, upload

pytestmark = pytest.mark.gpu


def test_graph_generations_match_direct_evaluation():
    n, n_cases = 500, 9000
    x = synth.uniform_cases(201, 1, n_cases)
    y = synth.quartic_target(x[0])
    pops = [synth.pack(synth.ramped_half_and_half(300 + g, n, 2, 8, 255)) for g in range(4)]
    max_tokens = max(int(p.lengths.sum()) for p in pops)
    gg = GenerationGraph(n, max_tokens, x, y)
    cfg = gp.Config(gp.VARIANT_REGISTER, 8, 256, 0)
    for pop in pops:
        got = gg.run(pop.words, pop.offsets, pop.lengths)
        enc = gp.encode_population(pop.words, pop.offsets, pop.lengths)
        P, O, L = upload(enc)
        ref = gp.eval_population(P, O, L, dev(x), dev(y), config=cfg).cpu().numpy()
        assert np.array_equal(got.view(np.uint64), ref.view(np.uint64))


def test_graph_rejects_a_population_too_large_for_its_capacity():
    x = synth.uniform_cases(202, 1, 1000)
    y = synth.quartic_target(x[0])
    small = synth.pack(synth.ramped_half_and_half(310, 64, 2, 3, 7))
    big = synth.pack(synth.ramped_half_and_half(311, 64, 6, 8, 255))
    gg = GenerationGraph(64, int(small.lengths.sum()), x, y)
    gg.run(small.words, small.offsets, small.lengths)
    with pytest.raises(ValueError):
        gg.run(big.words, big.offsets, big.lengths)
