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


@pytest.mark.parametrize("funcs,n_inputs,fitness", [(synth.FLOAT_FUNCS, 1, gp.FITNESS_SUM_ABS),
                                                    (synth.SHUTTLE_FUNCS, 9, gp.FITNESS_CLASS)])
def test_device_encoding_graph_matches_host_encoding(funcs, n_inputs, fitness):
    """The graph that copies the trees and encodes them on the device gives
    bit-identical fitness to host encoding, generation after generation (also
    for trees that are not packed back to back)."""
    n, n_cases = 300, 5000
    x = synth.uniform_cases(203, n_inputs, n_cases, -3.0, 3.0)
    y = np.rint(synth.uniform_cases(204, 1, n_cases, 0.0, 4.0)[0]).astype(np.float32)
    pops = [synth.pack(synth.ramped_half_and_half(320 + g, n, 1, 8, 255, funcs=funcs,
                                                  n_inputs=n_inputs, full_fallback_to_grow=True))
            for g in range(3)]
    max_tokens = max(int(p.lengths.sum()) for p in pops) + 64
    variant = gp.VARIANT_EXTENDED if funcs is synth.SHUTTLE_FUNCS else gp.VARIANT_REGISTER
    cfg = gp.Config(variant, 4, 128, 0, fitness)
    gh = GenerationGraph(n, max_tokens, x, y, config=cfg)
    gd = GenerationGraph(n, max_tokens, x, y, config=cfg, device_encode=True)
    for g, pop in enumerate(pops):
        words, offsets = pop.words, pop.offsets
        if g == 2:  # gaps between the trees
            words = np.zeros(pop.words.size + 2 * n, np.uint32)
            offsets = pop.offsets + 2 * np.arange(n)
            for p in range(n):
                words[offsets[p]: offsets[p] + pop.lengths[p]] = pop.program(p)
        a = gh.run(words, offsets, pop.lengths)
        b = gd.run(words, offsets, pop.lengths)
        assert np.array_equal(a.view(np.uint64), b.view(np.uint64)), g
    # layouts staged as they are (within the capacity): trees stored in
    # reverse order, and a one-word gap after every tenth tree
    pop = pops[1]
    rev = np.zeros(pop.words.size, np.uint32)
    roff = np.zeros(n, np.int64)
    pos = 0
    for p in reversed(range(n)):
        roff[p] = pos
        rev[pos: pos + pop.lengths[p]] = pop.program(p)
        pos += int(pop.lengths[p])
    gap = pop.offsets + np.arange(n) // 10
    gwords = np.zeros(pop.words.size + n // 10, np.uint32)
    for p in range(n):
        gwords[gap[p]: gap[p] + pop.lengths[p]] = pop.program(p)
    assert int(gap[-1] + pop.lengths[-1]) <= max_tokens
    for words, offsets in ((rev, roff), (gwords, gap)):
        a = gh.run(words, offsets, pop.lengths)
        b = gd.run(words, offsets, pop.lengths)
        assert np.array_equal(a.view(np.uint64), b.view(np.uint64))


@pytest.mark.parametrize("depth,device_encode", [(2, True), (3, False), (1, True)])
def test_pipeline_results_match_each_population(depth, device_encode):
    """Different populations submitted back to back through the pipeline's
    graphs: every ticket's fitness is that population's own (a result from
    another slot, or a slot overwritten before its copy finished, would
    differ), bit-identical to the direct evaluation, in submission order."""
    from paper_1601_00221_gb300.graph import EvaluationPipeline
    n, n_cases = 400, 7000
    x = synth.uniform_cases(205, 1, n_cases)
    y = synth.quartic_target(x[0])
    pops = [synth.pack(synth.ramped_half_and_half(340 + g, n, 2, 8, 255)) for g in range(7)]
    max_tokens = max(int(p.lengths.sum()) for p in pops)
    cfg = gp.Config(gp.VARIANT_REGISTER, 8, 256, 0)
    refs = []
    for pop in pops:
        enc = gp.encode_population(pop.words, pop.offsets, pop.lengths)
        P, O, L = upload(enc)
        refs.append(gp.eval_population(P, O, L, dev(x), dev(y), config=cfg).cpu().numpy())
    pipe = EvaluationPipeline(n, max_tokens, x, y, depth=depth, config=cfg, device_encode=device_encode)
    got = []
    for pop in pops:
        got += pipe.submit(pop.words, pop.offsets, pop.lengths)
        assert len(pipe.inflight) <= depth
    got += pipe.drain()
    assert [t for t, _ in got] == list(range(len(pops)))
    for t, fit in got:
        assert np.array_equal(fit.view(np.uint64), refs[t].view(np.uint64)), t
    assert pipe.drain() == []


def test_graph_launch_needs_collect():
    """A graph launched twice without collecting in between refuses: its
    pinned buffers still hold the launch in flight."""
    x = synth.uniform_cases(206, 1, 2000)
    y = synth.quartic_target(x[0])
    pop = synth.pack(synth.ramped_half_and_half(350, 64, 2, 6, 63))
    gg = GenerationGraph(64, int(pop.lengths.sum()), x, y)
    gg.launch(pop.words, pop.offsets, pop.lengths)
    with pytest.raises(RuntimeError):
        gg.launch(pop.words, pop.offsets, pop.lengths)
    first = gg.collect()
    with pytest.raises(RuntimeError):
        gg.collect()
    assert np.array_equal(first.view(np.uint64), gg.run(pop.words, pop.offsets, pop.lengths).view(np.uint64))
